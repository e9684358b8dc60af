"""The branch-and-bound lower bound is sound (never above the true narrowest
window at any candidate slope inside the interval) and exact on a point
interval; pinned by brute force over the candidate slopes (Sec. 3.1, 3.3)."""
from fractions import Fraction

import numpy as np

from oracle import bound, tiny


def test_bound_sound_and_tight():
    rng = np.random.default_rng(3)
    for trial in range(60):
        n = int(rng.integers(4, 14))
        xs = rng.integers(-50, 50, n).tolist()
        ys = rng.integers(-50, 50, n).tolist()
        h = n // 2 + 1
        pts = list(zip(xs, ys))
        S = tiny.candidate_slopes(pts)
        if len(S) < 2:
            continue
        i, j = sorted(rng.choice(len(S), 2, replace=False).tolist())
        a, b = S[i], S[j]
        lb = bound.lower_bound(xs, ys, h, a, b)
        inside = [s for s in S if a <= s <= b]
        assert lb <= min(bound.width_at(xs, ys, h, s) for s in inside)
        # and at any real slope of the interval
        for t in (Fraction(1, 3), Fraction(1, 2), Fraction(5, 7)):
            s = a + (b - a) * t
            assert lb <= bound.width_at(xs, ys, h, s)
        assert bound.lower_bound(xs, ys, h, a, a) == bound.width_at(xs, ys, h, a)
        assert lb >= 0


def test_bound_clamps_at_zero():
    # over a very wide slope interval the hulls of the projections overlap:
    # the difference of order statistics is negative and the bound is 0
    rng = np.random.default_rng(5)
    for _ in range(10):
        n = int(rng.integers(4, 12))
        xs = rng.integers(1, 50, n).tolist()          # x > 0: every hull is wide
        ys = rng.integers(-50, 50, n).tolist()
        h = n // 2 + 1
        assert bound.lower_bound(xs, ys, h, Fraction(-10**6), Fraction(10**6)) == 0


def test_width_matches_subset_definition():
    rng = np.random.default_rng(4)
    for _ in range(20):
        n = int(rng.integers(3, 8))
        xs = rng.integers(-9, 9, n).tolist()
        ys = rng.integers(-9, 9, n).tolist()
        s = Fraction(int(rng.integers(-20, 20)), int(rng.integers(1, 7)))
        h = n // 2 + 1
        assert bound.width_at(xs, ys, h, s) == tiny.window_width_at(list(zip(xs, ys)), h, s)[0]


def test_steep_bound_sound():
    # w(s) >= |s| dh - (y range) on each side of 0, pinned by the brute-force
    # window width at slopes of growing magnitude (exact rationals)
    rng = np.random.default_rng(6)
    for trial in range(40):
        n = int(rng.integers(4, 14))
        xs = rng.integers(-6, 6, n).tolist()          # repeated x: multiplicities above 1
        ys = rng.integers(-50, 50, n).tolist()
        h = n // 2 + 1
        dh = bound.span_lower_bound(xs, h)
        # dh is a true lower bound of the x span of every h-subset
        xsorted = sorted(xs)
        assert dh <= min(xsorted[k + h - 1] - xsorted[k] for k in range(n - h + 1))
        for smin in (Fraction(1, 2), Fraction(3), Fraction(40), Fraction(1000)):
            lb = bound.steep_lower_bound(xs, ys, h, smin)
            for s in (smin, smin * 2, smin + Fraction(1, 3)):
                assert lb <= bound.width_at(xs, ys, h, s)
                assert lb <= bound.width_at(xs, ys, h, -s)


def test_steep_bound_grows():
    # distinct x (m = 1): dh = h - 1 and the bound is positive for steep enough
    # slopes, so steep intervals can be pruned
    xs = list(range(10))
    ys = [3, -1, 4, 1, -5, 9, 2, -6, 5, 3]
    h = 6
    assert bound.span_lower_bound(xs, h) == 5
    assert bound.steep_lower_bound(xs, ys, h, Fraction(100)) == 100 * 5 - 15
