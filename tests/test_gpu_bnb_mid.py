"""Branch-and-bound above n = 8192, where the restricted pair pass is the
band scan over the points sorted at each cover's lower slope, the kept
events are re-bucketed from their own sample, the bounds sort 32-bit keys in
chunks (above 16384 points) and kept buckets may be refined into
sub-intervals: every result equals the plain sweep's bit for bit, on data
with large groups of equal slopes (a line of slope 0.7 with integer noise),
random slopes, collinear clusters (many points on a few exact lines, so
single slopes are shared by very many pairs, which also drives the plain
sweep's large-bucket fallback) and a narrow coordinate span (many repeated
x and whole duplicate points).  The sweep covers exactly the kept events (a
range lost or swept twice is LMS_ERR_INTERNAL)."""
import numpy as np
import pytest

from paper_1510_01041_gb300 import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

F = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j", "theta1", "theta2", "med_sq")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_01041_gb300 import build, lms
    build.build()
    return lms


def collinear_clusters(n, seed):
    """Points on four exact integer lines (slopes 1/3, -2, 5/4, 0) plus 30%
    uniform outliers: each line's points share one slope among all their
    pairs."""
    rng = np.random.default_rng(seed)
    m = n - int(0.3 * n)
    lines = [(1, 3, 100), (-2, 1, -50), (5, 4, 7), (0, 1, 300)]
    xs, ys = [], []
    for k in range(m):
        a, b, c = lines[k % 4]
        t = int(rng.integers(-2000, 2000))
        xs.append(b * t)
        ys.append(a * t + c)
    xs += rng.integers(-12000, 12000, n - m).tolist()
    ys += rng.integers(-12000, 12000, n - m).tolist()
    p = rng.permutation(n)
    return np.asarray(xs, np.int16)[p], np.asarray(ys, np.int16)[p]


def narrow_span(n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-60, 60, n).astype(np.int16), rng.integers(-60, 60, n).astype(np.int16)


CASES = [("line", 12288, 3), ("sloped", 9000, 4), ("sloped", 20000, 5), ("line", 20000, 6),
         ("clusters", 12000, 7), ("clusters", 24000, 8), ("narrow", 10000, 9)]


@pytest.mark.parametrize("gen,n,seed", CASES)
def test_bnb_equals_plain_sweep_above_8192(L, gen, n, seed):
    if gen == "line":
        x, y = datagen.line_with_outliers(n, seed, 0.4)
    elif gen == "sloped":
        x, y, _ = datagen.sloped(n, seed, 0.45, phi_max=1.4)
    elif gen == "clusters":
        x, y = collinear_clusters(n, seed)
    else:
        x, y = narrow_span(n, seed)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ref = L.decode(L.fit(xt, yt, 0, "sweep"))[0]
    assert ref["status"] == L.LMS_OK, (gen, n, ref)
    for mode in ("quantiles", "angles"):
        out, st = L.fit_bnb(xt, yt, 0, None, seed_mode=mode)
        r = L.decode(out)[0]
        assert {k: r[k] for k in F} == {k: ref[k] for k in F}, (gen, n, mode, r, ref)
        assert 0 < st["events_swept"] <= st["events_total"]
