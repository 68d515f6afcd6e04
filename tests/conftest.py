"""Shared test configuration. GPU tests carry ``@pytest.mark.gpu``."""
import pytest


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C-ABI library)")
