"""The oracle reproduces its stored fixtures (tests/golden/lms_small.json,
written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lms_small.json")
CASES = json.load(open(GOLD))["cases"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("method", ["brute", "sweep"])
def test_golden(orc, case, method):
    x = np.array(case["x"], dtype=np.int16)
    y = np.array(case["y"], dtype=np.int16)
    r = orc.lms_i16(x, y, case["h"], method)
    assert r.exact() == (case["status"], case["w_num"], case["w_den"], case["s_num"],
                         case["s_den"], case["t_num"], case["t_den"], case["i"], case["j"])
    assert (r.theta1, r.theta2, r.med_sq) == (case["theta1"], case["theta2"], case["med_sq"])
