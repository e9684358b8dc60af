"""Batched fits: every set's result equals the oracle bit for bit, with
plain-class and sweep sets mixed, per-set h, and a CUDA-graph replay."""
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


KEYS = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j", "theta1", "theta2", "med_sq")


def check(L, orc, x, y, off, res, h=None):
    for b in range(off.size - 1):
        xs, ys = x[off[b]:off[b + 1]], y[off[b]:off[b + 1]]
        hb = 0 if h is None else int(h[b])
        method = "brute" if xs.size <= 160 else "sweep"
        o = orc.lms_i16(xs, ys, hb, method)
        r = res[b]
        assert tuple(r[k] for k in KEYS) == tuple(getattr(o, k) for k in KEYS), (b, xs.size, r, o)


def test_batched_mixed_sizes(L, orc):
    x, y, off = datagen.batch(40, 3, n_min=2, n_max=1200)
    plan = L.BatchPlan(off, plain_max_n=256, streams=4)
    out = plan.fit(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(off).cuda())
    torch.cuda.synchronize()
    check(L, orc, x, y, off, L.decode(out))


def test_batched_degenerate_and_h(L, orc):
    rng = np.random.default_rng(5)
    xs, ys = [], []
    for k in range(30):
        n = int(rng.integers(2, 300))
        if k % 5 == 0:
            xv = np.full(n, 7)
        elif k % 5 == 1:
            xv = rng.integers(-2, 2, n)
        else:
            xv = rng.integers(-400, 400, n)
        xs.append(xv)
        ys.append(rng.integers(-400, 400, n))
    off = np.zeros(31, np.int64)
    off[1:] = np.cumsum([v.size for v in xs])
    x = np.concatenate(xs).astype(np.int16)
    y = np.concatenate(ys).astype(np.int16)
    h = np.array([[0, 1, 2, int(v.size)][k % 4] for k, v in enumerate(xs)], np.int32)
    h[h == 0] = [v.size // 2 + 1 for v in np.array(xs, dtype=object)[h == 0]]
    plan = L.BatchPlan(off, h=h, plain_max_n=128, streams=2)
    out = plan.fit(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(off).cuda())
    torch.cuda.synchronize()
    check(L, orc, x, y, off, L.decode(out), h)


def test_batched_graph_replay(L, orc):
    x, y, off = datagen.batch(24, 11, n_min=64, n_max=900)
    plan = L.BatchPlan(off, streams=4)
    xt, yt, ot = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(off).cuda()
    out = torch.zeros((24, L.RESULT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    plan.fit(xt, yt, ot, out=out)          # warm-up outside the capture
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(xt, yt, ot, out=out, stream=s)
    g.replay()
    torch.cuda.synchronize()
    check(L, orc, x, y, off, L.decode(out))
    # new data in the same buffers, replayed again
    x2, y2, _ = datagen.batch(24, 11, n_min=64, n_max=900)
    rng = np.random.default_rng(1)
    y2 = (y2.astype(np.int64) + rng.integers(-2, 3, y2.size)).clip(-32768, 32767).astype(np.int16)
    yt.copy_(torch.from_numpy(y2))
    g.replay()
    torch.cuda.synchronize()
    check(L, orc, x, y2, off, L.decode(out))


def test_batched_full_4096_sets_in_one_graph(L, orc):
    """The full batch workload: 4096 sets, n log-uniform in [64, 4096],
    outlier fraction U(0, 0.45), slope angle U(-1.5, 1.5), in the plan shape
    the benchmark tunes to (plain kernel up to 128 points, 48 streams),
    captured into one CUDA graph and replayed.  The smallest and largest sets
    and 30 random ones are checked against the oracle one by one; every set
    of the replay equals the eager run."""
    x, y, off = datagen.batch(4096, 5000)
    xt, yt, ot = (torch.from_numpy(a).cuda() for a in (x, y, off))
    plan = L.BatchPlan(off, plain_max_n=128, streams=48)
    out = plan.fit(xt, yt, ot)
    torch.cuda.synchronize()
    res = L.decode(out)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    out2 = torch.zeros_like(out)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(xt, yt, ot, out=out2, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), out2.cpu().numpy())
    sizes = np.diff(off)
    rng = np.random.default_rng(3)
    pick = sorted(set([int(np.argmin(sizes)), int(np.argmax(sizes))] + rng.choice(4096, 30, replace=False).tolist()))
    for b in pick:
        xs, ys = x[off[b]:off[b + 1]], y[off[b]:off[b + 1]]
        o = orc.lms_i16(xs, ys, 0, "brute" if xs.size <= 160 else "sweep")
        r = res[b]
        assert tuple(r[k] for k in KEYS) == tuple(getattr(o, k) for k in KEYS), (b, xs.size, r, o)
