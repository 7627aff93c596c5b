"""The oracle reproduces its frozen outputs on a fixed tiny problem
(tests/golden/oracle_tiny.json, written by tests/golden/make_golden.py from
oracle/ only): a change to the oracle's arithmetic fails here until the
fixture is regenerated on purpose."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402


def test_oracle_matches_frozen_outputs():
    want = json.load(open(os.path.join(HERE, "golden", "oracle_tiny.json")))
    got = make_golden.compute()
    assert np.allclose(got["I"], want["I"], rtol=1e-12, atol=0)
    for name in ("amplitude", "anscombe", "poisson", "gaussian", "epie"):
        for key, val in want[name].items():
            assert np.allclose(np.asarray(got[name][key]), np.asarray(val), rtol=1e-11, atol=1e-13), (name, key)
