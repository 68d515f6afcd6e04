"""CPU check of the force-region tile enumeration that the spread, the
region marking and the region check share: the host build of the same
header code visits exactly the tiles that hold a node of the box, for every
tile shape, on periodic and bounded axes, across the periodic seam and for
lattices smaller than a tile."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tile_enumeration_matches_brute_force(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "tile_cover_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "--expt-relaxed-constexpr", "-o", str(exe), os.path.join(HERE, "tile_cover_check.cu")],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout
