"""Exact branch-and-bound on the GPU: bit-identical to the oracle (and to
the plain sweep), with and without a seed slope; it prunes on typical data."""
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


F = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j", "theta1", "theta2", "med_sq")


def diff(r, o):
    return {k: (r[k], getattr(o, k)) for k in F if r[k] != getattr(o, k)}


def bnb(L, x, y, h=0, seed=None, mode="quantiles"):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    sd = None if seed is None else torch.tensor([seed], dtype=torch.float32, device="cuda")
    out, st = L.fit_bnb(xt, yt, h, sd, seed_mode=mode)
    torch.cuda.synchronize()
    return L.decode(out)[0], st


@pytest.mark.parametrize("n", [64, 300, 1024, 2048])
def test_bnb_matches_oracle(L, orc, n):
    for seed in range(3):
        x, y, meta = datagen.sloped(n, 40 + seed, 0.45, phi_max=1.4)
        o = orc.lms_i16(x, y, 0, "sweep")
        for sd in (None, float(np.tan(meta["phi"])), 3.0):
            r, st = bnb(L, x, y, 0, sd)
            assert not diff(r, o), (n, seed, sd, diff(r, o), st)
            assert st["events_swept"] <= st["events_total"]


def test_bnb_degenerate_and_h(L, orc):
    rng = np.random.default_rng(11)
    for trial in range(30):
        n = int(rng.integers(3, 90))
        span = int(rng.choice([4, 40, 3000]))
        x = rng.integers(-span, span, n).astype(np.int16)
        y = rng.integers(-span, span, n).astype(np.int16)
        h = [0, 1, n, int(rng.integers(1, n + 1))][trial % 4]
        r, _ = bnb(L, x, y, h, None)
        o = orc.lms_i16(x, y, h, "brute")
        assert not diff(r, o), (trial, n, h, diff(r, o))


@pytest.mark.parametrize("n", [700, 2048, 4096])
def test_bnb_scattered_survivors(L, orc, n):
    """A loose upper bound (evenly spaced angles) keeps many separated slope
    buckets: every sweeper must stay inside one run of kept buckets."""
    x, y, meta = datagen.sloped(n, 90 + n, 0.45, phi_max=1.4)
    o = orc.lms_i16(x, y, 0, "sweep")
    r, st = bnb(L, x, y, 0, None, "angles")
    assert not diff(r, o), (diff(r, o), st)
    r, st = bnb(L, x, y, 0, 2.5)          # a wrong prediction: still exact
    assert not diff(r, o), (diff(r, o), st)


def test_bnb_n8192_prunes_and_matches(L, orc):
    x, y, meta = datagen.sloped(8192, 7, 0.45, phi_max=1.4)
    o = orc.lms_i16(x, y, 0, "sweep")
    r, st = bnb(L, x, y, 0, float(np.tan(meta["phi"])))
    assert not diff(r, o), diff(r, o)
    assert st["events_swept"] < st["events_total"] // 4, st
    r2, st2 = bnb(L, x, y, 0, None)
    assert not diff(r2, o), diff(r2, o)


def test_bnb_equals_plain_sweep_on_many_instances(L):
    """Both workload generators at n = 2048 .. 8192 over many seeds (fixed
    slope 0.7 with its large equal-slope groups; random slopes with up to 45%
    outliers): every seeding of the branch-and-bound (sample quantiles,
    evenly spaced angles, a wildly wrong predicted slope) returns the plain
    sweep's result bit for bit, and the sweep covers exactly the kept
    events (a range left out is reported as LMS_ERR_INTERNAL)."""
    cases = [("line", 8192, s, 0.4) for s in range(1, 25)]
    cases += [("sloped", n, 500 + s, f) for s in range(12) for n, f in ((2048, 0.3), (8192, 0.45))]
    for gen, n, seed, frac in cases:
        if gen == "line":
            x, y = datagen.line_with_outliers(n, seed, frac)
        else:
            x, y, _ = datagen.sloped(n, seed, frac, phi_max=1.4)
        xt = torch.from_numpy(x).cuda()
        yt = torch.from_numpy(y).cuda()
        ref = L.decode(L.fit(xt, yt, 0, "sweep"))[0]
        assert ref["status"] == L.LMS_OK, (gen, n, seed)
        for mode, sd in (("quantiles", None), ("angles", None), ("quantiles", 40.0)):
            r, st = bnb(L, x, y, 0, sd, mode)
            assert {k: r[k] for k in F} == {k: ref[k] for k in F}, (gen, n, seed, mode, sd, r, ref)
            assert st["events_swept"] <= st["events_total"]
