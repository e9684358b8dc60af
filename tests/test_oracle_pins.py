"""Pins for the CPU oracle against facts fixed by the paper and by mathematics,
not against the oracle itself.  No GPU needed.

* exhaustive subset search on tiny inputs (definition, Sec. 1 Eq. 1, Sec. 3.1)
* half the points in a slab: minimax fits of h-subsets (Sec. 3.1)
* the equioscillation property (Sec. 3.3): the optimum equals the best
  triple-equioscillating line
* the candidate set (Sec. 3.3, 3.4.1): no real slope beats the pairwise slopes
* zero residual when h points are collinear (Sec. 3.1, slab of height 0)
* regression, scale and affine equivariance (Sec. 1)
* h = n: the Chebyshev line, checked against a linear program (scipy HiGHS)
* permutation invariance and a residual certificate of the returned line
* O1 (brute force) and O2 (sweep, Sec. 2) agree bit for bit
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import tiny
from paper_1510_01041_gb300 import datagen


def _frac(r):
    return (Fraction(r.w_num, r.w_den), Fraction(r.s_num, r.s_den),
            Fraction(r.t_num, r.t_den))


def _random_small(rng, n, span):
    x = rng.integers(-span, span, n).astype(np.int16)
    y = rng.integers(-span, span, n).astype(np.int16)
    return x, y


def _degenerate(rng, n):
    """Duplicates, collinear runs and repeated x values."""
    kind = rng.integers(0, 4)
    if kind == 0:
        x, y = _random_small(rng, n, 3)
    elif kind == 1:          # several points on one line plus noise points
        k = max(2, n // 2)
        xs = rng.integers(-5, 5, k)
        x = np.concatenate([xs, rng.integers(-9, 9, n - k)])
        y = np.concatenate([2 * xs + 1, rng.integers(-9, 9, n - k)])
    elif kind == 2:          # duplicated points
        x, y = _random_small(rng, n, 6)
        m = n // 2
        x[:m] = x[m:2 * m]
        y[:m] = y[m:2 * m]
    else:                    # few distinct x values
        x = rng.integers(-2, 2, n)
        y = rng.integers(-50, 50, n)
    return x.astype(np.int16), y.astype(np.int16)


def test_o1_equals_exhaustive_subsets(orc):
    rng = np.random.default_rng(20251)
    checked = 0
    for trial in range(320):
        n = int(rng.integers(2, 9))
        if trial % 2:
            x, y = _degenerate(rng, n)
        else:
            x, y = _random_small(rng, n, int(rng.choice([4, 30, 20000])))
        h = int(rng.integers(1, n + 1)) if trial % 3 == 0 else n // 2 + 1
        r = orc.lms_i16(x, y, h, "brute")
        t = tiny.lms_subsets(list(zip(x.tolist(), y.tolist())), h)
        if t is None:
            assert r.status == orc.ERR_VERTICAL
            continue
        w, s, c, pair = t
        assert r.status == orc.OK
        assert _frac(r) == (w, s, c), (x, y, h)
        assert (r.i, r.j) == pair
        checked += 1
    assert checked > 250


def test_value_equals_best_subset_chebyshev_fit(orc):
    rng = np.random.default_rng(7)
    for trial in range(60):
        n = int(rng.integers(3, 9))
        x, y = _random_small(rng, n, 50) if trial % 2 else _degenerate(rng, n)
        if len(set(x.tolist())) < 2:
            continue
        h = n // 2 + 1
        r = orc.lms_i16(x, y, h, "brute")
        v = tiny.lms_chebyshev(list(zip(x.tolist(), y.tolist())), h)
        assert Fraction(r.w_num, 2 * r.w_den) == v


def test_equioscillation_triple(orc):
    """Sec. 3.3: the LMS line equioscillates w.r.t. some triple of points; every
    triple's equioscillating line is a feasible line, so min over triples of its
    h-th smallest |residual| equals the LMS value (general position)."""
    rng = np.random.default_rng(11)
    done = 0
    while done < 40:
        n = int(rng.integers(4, 9))
        x = rng.choice(np.arange(-200, 200), n, replace=False).astype(np.int16)
        y = rng.integers(-200, 200, n).astype(np.int16)
        pts = list(zip(x.tolist(), y.tolist()))
        slopes = [Fraction(b[1] - a[1], b[0] - a[0]) for k, a in enumerate(pts) for b in pts[k + 1:]]
        if len(set(slopes)) != len(slopes):
            continue          # keep general position: no two parallel pairs
        r = orc.lms_i16(x, y, 0, "brute")
        assert tiny.lms_equioscillation(pts) == Fraction(r.w_num, 2 * r.w_den)
        done += 1
    # feasibility alone holds on any input
    for _ in range(30):
        n = int(rng.integers(3, 9))
        x, y = _degenerate(rng, n)
        v = tiny.lms_equioscillation(list(zip(x.tolist(), y.tolist())))
        if v is not None:
            r = orc.lms_i16(x, y, 0, "brute")
            assert v >= Fraction(r.w_num, 2 * r.w_den)


def test_no_real_slope_is_better(orc):
    rng = np.random.default_rng(5)
    for _ in range(25):
        n = int(rng.integers(3, 8))
        x, y = _random_small(rng, n, 40)
        if len(set(x.tolist())) < 2:
            continue
        h = n // 2 + 1
        r = orc.lms_i16(x, y, h, "brute")
        wstar = Fraction(r.w_num, r.w_den)
        pts = list(zip(x.tolist(), y.tolist()))
        for _ in range(12):
            s = Fraction(int(rng.integers(-4000, 4000)), int(rng.integers(1, 997)))
            w, _ = tiny.window_width_at(pts, h, s)
            assert w >= wstar


@pytest.mark.parametrize("seed", range(6))
def test_zero_residual_when_h_collinear(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(7, 60))
    h = n // 2 + 1
    p, q, c = int(rng.integers(-5, 6)), int(rng.integers(1, 5)), int(rng.integers(-50, 50))
    xs = rng.choice(np.arange(-400, 400), h, replace=False) * q
    ys = (xs // q) * p + c
    xo = rng.integers(-3000, 3000, n - h)
    yo = rng.integers(-3000, 3000, n - h)
    x = np.concatenate([xs, xo]).astype(np.int16)
    y = np.concatenate([ys, yo]).astype(np.int16)
    perm = rng.permutation(n)
    r = orc.lms_i16(x[perm], y[perm], h, "sweep")
    assert r.w_num == 0 and r.med_sq == 0.0
    assert Fraction(r.s_num, r.s_den) == Fraction(p, q)
    assert Fraction(r.t_num, r.t_den) == c


def _unique_optimum(orc, x, y, h):
    """True if exactly one (slope, centre) attains the minimum width."""
    r = orc.lms_i16(x, y, h, "brute")
    w = Fraction(r.w_num, r.w_den)
    pts = list(zip(x.tolist(), y.tolist()))
    hits = set()
    for s in tiny.candidate_slopes(pts):
        ww, c = tiny.window_width_at(pts, h, s)
        if ww == w:
            hits.add(s)
    return len(hits) == 1


def test_regression_equivariance(orc):
    """y -> y + a x + b gives theta1 + a, theta2 + b, the same slab height."""
    rng = np.random.default_rng(3)
    for trial in range(40):
        n = int(rng.integers(5, 40))
        x, y = _random_small(rng, n, 200)
        a, b = int(rng.integers(-3, 4)), int(rng.integers(-100, 100))
        y2 = (y.astype(np.int64) + a * x + b).astype(np.int16)
        r1 = orc.lms_i16(x, y, 0, "sweep")
        r2 = orc.lms_i16(x, y2, 0, "sweep")
        assert Fraction(r1.w_num, r1.w_den) == Fraction(r2.w_num, r2.w_den)
        # the slope order is preserved by a shear, so the tie-break is too
        assert Fraction(r2.s_num, r2.s_den) == Fraction(r1.s_num, r1.s_den) + a
        assert Fraction(r2.t_num, r2.t_den) == Fraction(r1.t_num, r1.t_den) + b


def test_scale_equivariance(orc):
    """y -> c y (c > 0) scales theta by c and med_sq by c^2; x -> c x + d (c > 0)
    maps theta1 -> theta1 / c, theta2 -> theta2 - theta1 d / c."""
    rng = np.random.default_rng(4)
    for trial in range(40):
        n = int(rng.integers(5, 40))
        x, y = _random_small(rng, n, 300)
        c = int(rng.integers(2, 9))
        r1 = orc.lms_i16(x, y, 0, "sweep")
        ry = orc.lms_i16(x, (y.astype(np.int64) * c).astype(np.int16), 0, "sweep")
        assert Fraction(ry.w_num, ry.w_den) == c * Fraction(r1.w_num, r1.w_den)
        assert Fraction(ry.s_num, ry.s_den) == c * Fraction(r1.s_num, r1.s_den)
        assert Fraction(ry.t_num, ry.t_den) == c * Fraction(r1.t_num, r1.t_den)
        d = int(rng.integers(-500, 500))
        rx = orc.lms_i16((x.astype(np.int64) * c + d).astype(np.int16), y, 0, "sweep")
        assert Fraction(rx.w_num, rx.w_den) == Fraction(r1.w_num, r1.w_den)
        s1 = Fraction(r1.s_num, r1.s_den)
        assert Fraction(rx.s_num, rx.s_den) == s1 / c
        assert Fraction(rx.t_num, rx.t_den) == Fraction(r1.t_num, r1.t_den) - s1 * d / c


def test_mirror_keeps_value(orc):
    """x -> -x reverses the slope order: the slab height is unchanged, and the
    line maps to (-theta1, theta2) whenever the optimum is unique."""
    rng = np.random.default_rng(9)
    for trial in range(30):
        n = int(rng.integers(4, 8))
        x, y = _random_small(rng, n, 100)
        r1 = orc.lms_i16(x, y, 0, "brute")
        r2 = orc.lms_i16(-x, y, 0, "brute")
        assert Fraction(r1.w_num, r1.w_den) == Fraction(r2.w_num, r2.w_den)
        if r1.status == 0 and _unique_optimum(orc, x, y, n // 2 + 1):
            assert Fraction(r2.s_num, r2.s_den) == -Fraction(r1.s_num, r1.s_den)
            assert Fraction(r2.t_num, r2.t_den) == Fraction(r1.t_num, r1.t_den)


def test_h_equals_n_is_chebyshev_lp(orc):
    """h = n: the slab must hold every point, i.e. the minimax line; solve the
    linear program min t s.t. |y_k - a x_k - b| <= t with scipy's HiGHS."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    rng = np.random.default_rng(12)
    for _ in range(20):
        n = int(rng.integers(3, 80))
        x, y = _random_small(rng, n, 1000)
        if len(set(x.tolist())) < 2:
            continue
        r = orc.lms_i16(x, y, n, "sweep")
        X = x.astype(float)
        Y = y.astype(float)
        A = np.vstack([np.column_stack([-X, -np.ones(n), -np.ones(n)]),
                       np.column_stack([X, np.ones(n), -np.ones(n)])])
        bvec = np.concatenate([-Y, Y])
        lp = linprog([0, 0, 1], A_ub=A, b_ub=bvec, bounds=[(None, None)] * 3, method="highs")
        assert lp.status == 0
        assert abs(lp.fun - r.w_num / (2 * r.w_den)) <= 1e-7 * max(1.0, lp.fun)


def test_h_one_is_zero(orc):
    x, y = datagen.line_with_outliers(40, 3)
    r = orc.lms_i16(x, y, 1, "sweep")
    assert r.w_num == 0 and r.status == 0


def test_permutation_invariance(orc):
    x, y = datagen.line_with_outliers(300, 21)
    r1 = orc.lms_i16(x, y, 0, "sweep")
    perm = datagen.Stream(99).permutation(300)
    r2 = orc.lms_i16(x[perm], y[perm], 0, "sweep")
    assert r1.exact()[:7] == r2.exact()[:7]
    assert (r1.theta1, r1.theta2, r1.med_sq) == (r2.theta1, r2.theta2, r2.med_sq)


def test_certificate_hth_residual(orc):
    """The returned line's h-th smallest |residual| is exactly w/2:
    |2 sd r_k| = |2 sd y_k - 2 sn x_k - t_num|."""
    for seed in range(4):
        x, y = datagen.line_with_outliers(257 + 40 * seed, seed)
        n = x.size
        h = n // 2 + 1
        r = orc.lms_i16(x, y, 0, "sweep")
        res = np.abs(2 * r.s_den * y.astype(np.int64) - 2 * r.s_num * x.astype(np.int64) - r.t_num)
        assert np.sort(res)[h - 1] == r.w_num


def test_vertical_input(orc):
    x = np.full(9, 17, dtype=np.int16)
    y = np.arange(9, dtype=np.int16) * 3
    for m in ("brute", "sweep"):
        r = orc.lms_i16(x, y, 0, m)
        assert r.status == orc.ERR_VERTICAL
        assert r.w_num == 12 and r.s_num == 0 and r.s_den == 1


def test_bad_arguments(orc):
    r = orc.lms_i16(np.zeros(1, np.int16), np.zeros(1, np.int16), 0, "brute")
    assert r.status == orc.ERR_ARG
    r = orc.lms_i16(np.arange(5, dtype=np.int16), np.arange(5, dtype=np.int16), 6, "sweep")
    assert r.status == orc.ERR_ARG


@pytest.mark.parametrize("gen", ["line", "sloped", "dense", "collinear"])
def test_brute_equals_sweep(orc, gen):
    rng = np.random.default_rng({"line": 1, "sloped": 2, "dense": 3, "collinear": 4}[gen])
    for trial in range(6):
        n = int(rng.integers(20, 260))
        if gen == "line":
            x, y = datagen.line_with_outliers(n, trial)
        elif gen == "sloped":
            x, y, _ = datagen.sloped(n, trial, 0.3)
        elif gen == "dense":
            x, y = _random_small(rng, n, 6)
        else:
            k = n // 2
            xs = rng.integers(-30, 30, k)
            x = np.concatenate([xs, rng.integers(-40, 40, n - k)]).astype(np.int16)
            y = np.concatenate([3 * xs - 2, rng.integers(-40, 40, n - k)]).astype(np.int16)
        h = [0, 2, n // 3 + 1, n][trial % 4]
        assert orc.lms_i16(x, y, h, "brute").exact() == orc.lms_i16(x, y, h, "sweep").exact()


def test_recovery_sanity(orc):
    """Not parity: with 40% outliers the LMS line sits on the generating line."""
    x, y = datagen.line_with_outliers(512, 1)
    r = orc.lms_i16(x, y, 0, "sweep")
    assert abs(r.theta1 - 0.7) < 0.01 and abs(r.theta2 - 100.0) < 8


def test_float_oracle(orc):
    # integer-valued floats give the integer path's numbers exactly
    x, y = datagen.line_with_outliers(120, 8)
    ri = orc.lms_i16(x, y, 0, "sweep")
    rf = orc.lms_f32(x.astype(np.float32), y.astype(np.float32), 0, "sweep")
    assert (ri.theta1, ri.theta2, ri.med_sq) == (rf.theta1, rf.theta2, rf.med_sq)
    # brute force and sweep agree on general floats; power-of-two scaling is exact
    xf, yf = datagen.gaussian_f32(150, 2)
    a = orc.lms_f32(xf, yf, 0, "brute")
    b = orc.lms_f32(xf, yf, 0, "sweep")
    assert (a.theta1, a.theta2, a.med_sq, a.i, a.j) == (b.theta1, b.theta2, b.med_sq, b.i, b.j)
    c = orc.lms_f32(xf * np.float32(8), yf * np.float32(8), 0, "sweep")
    assert c.med_sq == 64 * b.med_sq and c.theta1 == b.theta1


def _float_small(rng, n, trial):
    """Tiny float32 sets with fractional bits: spread exponents, dyadic
    grids with duplicates and repeated x, and exact float lines."""
    kind = trial % 4
    if kind == 0:
        x = rng.standard_normal(n) * 2.0 ** rng.integers(-6, 7, n)
        y = rng.standard_normal(n) * 2.0 ** rng.integers(-6, 7, n)
    elif kind == 1:
        x = rng.integers(-12, 12, n) / 8.0
        y = rng.integers(-40, 40, n) / 16.0
        m = n // 2
        x[:m] = x[n - m:]
    elif kind == 2:
        x = rng.integers(-3, 3, n) * 0.375
        y = rng.standard_normal(n) * 10.0
    else:
        x = rng.integers(-20, 20, n) / 4.0
        y = 0.5 * x + 0.25
        k = n // 3
        y[:k] = rng.standard_normal(k) * 4.0
    return x.astype(np.float32), y.astype(np.float32)


@pytest.mark.parametrize("method", ["brute", "sweep"])
def test_float_oracle_equals_exhaustive_subsets(orc, method):
    """The float path (coordinates scaled by 2^scale_exp into exact integers)
    against the definition in exact rationals on the float values as given
    (Sec. 1 Eq. 1, Sec. 3.1): the pair exactly; the width, slope and centre
    exactly where they fit the result's int64 fields (which hold 0 when they
    do not); and the reported doubles within the roundings of their
    conversion (the 128-bit numerator and denominator each rounded to double,
    one division, and for med_sq one product)."""
    rng = np.random.default_rng(4242)
    checked = exact = 0
    for trial in range(160):
        n = int(rng.integers(2, 9))
        x, y = _float_small(rng, n, trial)
        h = int(rng.integers(1, n + 1)) if trial % 3 == 0 else n // 2 + 1
        r = orc.lms_f32(x, y, h, method)
        pts = [(Fraction(float(a)), Fraction(float(b))) for a, b in zip(x, y)]
        t = tiny.lms_subsets(pts, h)
        if t is None:
            assert r.status == orc.ERR_VERTICAL
            continue
        w, s, c, pair = t
        assert r.status == orc.OK
        assert (r.i, r.j) == pair, (x, y, h)
        if r.s_den:
            sc = Fraction(2) ** r.scale_exp
            got = (Fraction(r.w_num, r.w_den) / sc, Fraction(r.s_num, r.s_den), Fraction(r.t_num, r.t_den) / sc)
            assert got == (w, s, c), (x, y, h)
            exact += 1
        u = 2.0 ** -53
        assert abs(r.theta1 - float(s)) <= 4 * u * abs(float(s))
        assert abs(r.theta2 - float(c)) <= 4 * u * abs(float(c))
        assert abs(r.med_sq - float((w / 2) ** 2)) <= 8 * u * float((w / 2) ** 2)
        checked += 1
    assert checked > 120 and exact > 80


def test_eval_slope_equals_subset_window(orc):
    """The oracle's window at a given rational slope (used by the large-size
    certificate tests) equals the definition by subsets at that slope: the
    narrowest range of h projections and the smallest centre among the
    narrowest (Sec. 3.1), for reduced and unreduced slopes, h = 1 .. n."""
    rng = np.random.default_rng(99)
    for trial in range(300):
        n = int(rng.integers(1, 9))
        x, y = _random_small(rng, n, int(rng.choice([3, 30, 30000])))
        h = int(rng.integers(1, n + 1))
        sd = int(rng.integers(1, 40))
        sn = int(rng.integers(-200, 201)) if trial % 5 else int(rng.integers(-40000, 40001))
        k = int(rng.integers(1, 4))
        r = orc.eval_slope_i16(x, y, sn * k, sd * k, h)
        assert r.status == orc.OK
        w, c = tiny.window_width_at(list(zip(x.tolist(), y.tolist())), h, Fraction(sn, sd))
        assert Fraction(r.w_num, r.w_den) == w, (x, y, h, sn, sd)
        assert Fraction(r.t_num, r.t_den) == c, (x, y, h, sn, sd)
        assert Fraction(r.s_num, r.s_den) == Fraction(sn, sd)
