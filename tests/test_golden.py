"""The oracle still reproduces its committed regression record
(``tests/golden/oracle_small_shear.json``, written by
``tests/golden/make_golden.py`` from the oracle alone)."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.join(os.path.dirname(__file__), "golden")


def test_oracle_matches_its_record():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(HERE, "oracle_small_shear.json")) as fh:
        ref = json.load(fh)
    got = mod.record()
    for k, v in ref.items():
        if isinstance(v, str):
            assert got[k] == v
        else:
            assert np.allclose(got[k], v, rtol=1e-12, atol=1e-18), k
