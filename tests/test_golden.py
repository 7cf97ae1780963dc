"""The oracle still reproduces its committed regression record (written by
tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_golden_record(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    want = json.load(open(os.path.join(HERE, "golden", "tiny_march.json")))
    got = mk.record()
    assert got["seed_iters"] == want["seed_iters"]
    assert np.allclose(got["seed"], want["seed"], rtol=1e-12, atol=0)
    assert np.allclose(got["targets"], want["targets"], rtol=1e-12, atol=0)
