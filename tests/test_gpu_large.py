"""Exact fits at n = 65536 (int16, 45% outliers: the branch-and-bound
configuration of the largest workload).  At this size the sweep keeps each
warp's position array in global memory (order and positions no longer fit
in shared memory together) and every bucket is sorted by chunk sorts plus
merges.  The full oracle sweep would take minutes on the host, so the check
is by properties that hold at any size:

* the branch-and-bound and the plain sweep (every candidate slope) agree
  bit for bit;
* certificate: the oracle's narrowest window at the reported slope is the
  reported window (width, centre) exactly;
* no other candidate slope the oracle evaluates (pairs through the reported
  window's region and random pairs) has a narrower window.
"""
import numpy as np
import pytest

from paper_1510_01041_gb300 import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_01041_gb300 import build, lms
    build.build()
    return lms


def _fit(L, x, y, algorithm):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = L.fit(xt, yt, 0, algorithm)
    torch.cuda.synchronize()
    return L.decode(out)[0]


KEYS = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j", "theta1", "theta2", "med_sq")


def test_n65536_branch_and_bound_equals_sweep_with_certificate(L, orc):
    n = 65536
    x, y = datagen.line_with_outliers(n, 11, 0.45)
    rb = _fit(L, x, y, "bnb")
    rs = _fit(L, x, y, "sweep")
    assert rb["status"] == L.LMS_OK
    assert tuple(rb[k] for k in KEYS) == tuple(rs[k] for k in KEYS)
    # the reported slope's narrowest window, exactly
    c = orc.eval_slope_i16(x, y, int(rb["s_num"]), int(rb["s_den"]), 0)
    assert (c.w_num, c.w_den) == (rb["w_num"], rb["w_den"])
    assert (c.t_num, c.t_den) == (rb["t_num"], rb["t_den"])
    # no evaluated candidate slope does better (width compared as exact rationals)
    rng = np.random.default_rng(5)
    xi, yi = x.astype(np.int64), y.astype(np.int64)
    pairs = [(int(rb["i"]), int(rb["j"]))]
    pairs += [tuple(int(v) for v in rng.choice(n, 2, replace=False)) for _ in range(24)]
    # pairs among points close to the reported line (where competitors live)
    resid = np.abs(yi * int(rb["s_den"]) - xi * int(rb["s_num"]) - 0)
    near = np.argsort(resid - np.median(resid))[: 2000]
    pairs += [tuple(int(v) for v in rng.choice(near, 2, replace=False)) for _ in range(24)]
    W, D = int(rb["w_num"]), int(rb["w_den"])
    for i, j in pairs:
        dx, dy = int(xi[j] - xi[i]), int(yi[j] - yi[i])
        if dx == 0:
            continue
        if dx < 0:
            dx, dy = -dx, -dy
        e = orc.eval_slope_i16(x, y, dy, dx, 0)
        assert e.w_num * D >= W * e.w_den, (i, j, e.w_num, e.w_den, W, D)
