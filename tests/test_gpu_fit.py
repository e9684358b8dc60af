"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer inputs must match bit for bit: status, the exact rationals
(w, theta1, theta2), the index pair and the three doubles.
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


def gpu_fit(L, x, y, h=0, algorithm="auto", **kw):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = L.fit(xt, yt, h, algorithm, **kw)
    torch.cuda.synchronize()
    return L.decode(out)[0]


FIELDS = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j",
          "theta1", "theta2", "med_sq")


class Diff:
    """Truthy when the GPU record equals the oracle's; repr lists the differences."""

    def __init__(self, r, o):
        self.d = {k: (r[k], getattr(o, k)) for k in FIELDS if r[k] != getattr(o, k)}

    def __bool__(self):
        return not self.d

    def __repr__(self):
        return "differs (gpu, oracle): " + repr(self.d)


def same(r, o):
    return Diff(r, o)


def _degenerate(rng, n):
    kind = int(rng.integers(0, 4))
    if kind == 0:
        x = rng.integers(-3, 3, n); y = rng.integers(-3, 3, n)
    elif kind == 1:
        k = max(2, n // 2)
        xs = rng.integers(-40, 40, k)
        x = np.concatenate([xs, rng.integers(-90, 90, n - k)])
        y = np.concatenate([2 * xs + 1, rng.integers(-90, 90, n - k)])
    elif kind == 2:
        x = rng.integers(-30, 30, n); y = rng.integers(-30, 30, n)
        m = n // 2
        x[:m] = x[m:2 * m]; y[:m] = y[m:2 * m]
    else:
        x = rng.integers(-2, 2, n); y = rng.integers(-500, 500, n)
    return x.astype(np.int16), y.astype(np.int16)


@pytest.mark.parametrize("algorithm", ["plain", "sweep", "paper"])
def test_small_random_and_degenerate(L, orc, algorithm):
    rng = np.random.default_rng({"plain": 77, "sweep": 78, "paper": 79}[algorithm])
    for trial in range(60):
        n = int(rng.integers(2, 70))
        if trial % 2:
            x, y = _degenerate(rng, n)
        else:
            span = int(rng.choice([5, 100, 16000]))
            x = rng.integers(-span, span, n).astype(np.int16)
            y = rng.integers(-span, span, n).astype(np.int16)
        h = [0, 1, n, int(rng.integers(1, n + 1))][trial % 4]
        r = gpu_fit(L, x, y, h, algorithm)
        o = orc.lms_i16(x, y, h, "brute")
        assert same(r, o), (algorithm, trial, n, h, r, o)


def test_full_int16_range_uses_int64_keys(L, orc):
    rng = np.random.default_rng(5)
    for trial in range(6):
        n = int(rng.integers(40, 300))
        x = rng.integers(-32768, 32768, n).astype(np.int16)
        y = rng.integers(-32768, 32768, n).astype(np.int16)
        o = orc.lms_i16(x, y, 0, "sweep")
        for algo in ("plain", "sweep"):
            assert same(gpu_fit(L, x, y, 0, algo), o), (trial, algo)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_plain_config_n512(L, orc, seed):
    """Single plain instance, n = 512, 40% outliers (all 130,816 slopes)."""
    x, y = datagen.line_with_outliers(512, seed)
    o = orc.lms_i16(x, y, 0, "brute")
    assert same(gpu_fit(L, x, y, 0, "plain"), o)
    assert same(gpu_fit(L, x, y, 0, "sweep"), o)
    assert same(gpu_fit(L, x, y, 0, "paper"), o)


@pytest.mark.parametrize("n", [128, 256, 300, 1024])
def test_paper_layout_table1_sizes(L, orc, n):
    """The paper's own kernel layout (8 x 8 vertex blocks, a thread block and a
    bitonic sort per vertex) at the sizes of its Table 1, a size that is not a
    power of two (padding) and its largest supported size."""
    x, y = datagen.line_with_outliers(n, 40 + n)
    o = orc.lms_i16(x, y, 0, "brute")
    assert same(gpu_fit(L, x, y, 0, "paper"), o)
    xs, ys, _ = datagen.sloped(n, 50 + n, 0.3)
    o = orc.lms_i16(xs, ys, 0, "brute")
    assert same(gpu_fit(L, xs, ys, 0, "paper"), o)


@pytest.mark.parametrize("n", [300, 777, 1024, 2048])
def test_sweep_matches_oracle_sweep(L, orc, n):
    for seed in range(2):
        x, y = datagen.line_with_outliers(n, 10 + seed)
        o = orc.lms_i16(x, y, 0, "sweep")
        assert same(gpu_fit(L, x, y, 0, "sweep"), o), (n, seed)
        xs, ys, _ = datagen.sloped(n, 20 + seed, 0.3)
        o = orc.lms_i16(xs, ys, 0, "sweep")
        assert same(gpu_fit(L, xs, ys, 0, "sweep"), o), (n, seed, "sloped")


def test_sweep_heavy_collinear(L, orc):
    """Large groups of equal slopes: many points on few lattice lines."""
    rng = np.random.default_rng(9)
    n = 1500
    k = 700
    xs = rng.integers(-200, 200, k)
    x = np.concatenate([xs, rng.integers(-300, 300, n - k)]).astype(np.int16)
    y = np.concatenate([xs // 2 * 2 + (xs % 3), rng.integers(-300, 300, n - k)]).astype(np.int16)
    o = orc.lms_i16(x, y, 0, "sweep")
    assert same(gpu_fit(L, x, y, 0, "sweep"), o)


def test_sweep_n8192(L, orc):
    x, y = datagen.line_with_outliers(8192, 1)
    o = orc.lms_i16(x, y, 0, "sweep")
    assert same(gpu_fit(L, x, y, 0, "sweep"), o)


def test_sweep_n16384(L, orc):
    """n above the shared-memory start sort; buckets above the shared-memory
    segment cap are sorted by chunk sorts plus merges."""
    x, y = datagen.line_with_outliers(16384, 2)
    o = orc.lms_i16(x, y, 0, "sweep")
    assert same(gpu_fit(L, x, y, 0, "sweep"), o)


def test_oversize_buckets_merge(L, orc):
    """Few buckets: every bucket is far above the shared-memory cap, so the
    events go through the chunk sorts and several merge rounds."""
    x, y = datagen.line_with_outliers(2048, 7)
    o = orc.lms_i16(x, y, 0, "sweep")
    for bk in (1, 5, 33):
        assert same(gpu_fit(L, x, y, 0, "sweep", buckets=bk), o), bk
    rng = np.random.default_rng(19)
    k = 900
    xs = rng.integers(-300, 300, k)
    xc = np.concatenate([xs, rng.integers(-400, 400, 2000 - k)]).astype(np.int16)
    yc = np.concatenate([3 * xs - 7, rng.integers(-900, 900, 2000 - k)]).astype(np.int16)
    o = orc.lms_i16(xc, yc, 0, "sweep")
    for bk in (2, 9):
        assert same(gpu_fit(L, xc, yc, 0, "sweep", buckets=bk), o), ("collinear", bk)


def test_sweeper_and_bucket_counts_do_not_change_result(L, orc):
    x, y = datagen.line_with_outliers(1500, 4)
    o = orc.lms_i16(x, y, 0, "sweep")
    for sw, bk in ((1, 1), (7, 3), (64, 200), (1000, 2000)):
        assert same(gpu_fit(L, x, y, 0, "sweep", sweepers=sw, buckets=bk), o), (sw, bk)


def test_vertical_and_tiny(L, orc):
    x = np.full(9, 17, np.int16)
    y = (np.arange(9) * 3).astype(np.int16)
    for algo in ("plain", "sweep"):
        r = gpu_fit(L, x, y, 0, algo)
        assert same(r, orc.lms_i16(x, y, 0, "brute"))
        assert r["status"] == L.LMS_ERR_VERTICAL
    x2 = np.array([0, 5], np.int16)
    y2 = np.array([1, -4], np.int16)
    for algo in ("plain", "sweep"):
        assert same(gpu_fit(L, x2, y2, 0, algo), orc.lms_i16(x2, y2, 0, "brute"))


def test_host_entry_point(L, orc):
    x, y = datagen.line_with_outliers(600, 6)
    r = L.fit_host(x, y, 0, "sweep")
    assert same(r, orc.lms_i16(x, y, 0, "sweep"))


def test_permutation_invariance_gpu(L):
    x, y = datagen.line_with_outliers(3000, 12)
    p = datagen.Stream(5).permutation(3000)
    a = gpu_fit(L, x, y, 0, "sweep")
    b = gpu_fit(L, x[p], y[p], 0, "sweep")
    for k in ("w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "theta1", "theta2", "med_sq"):
        assert a[k] == b[k]
