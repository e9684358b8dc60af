"""Branch-and-bound bound oracle (exact rationals, pure Python/numpy).

TEST INFRASTRUCTURE ONLY.  For a slope interval [a, b] every projection
z_k(s) = y_k - s x_k is linear in s, so it lies between
lo_k = min(z_k(a), z_k(b)) and hi_k = max(z_k(a), z_k(b)) on the interval.
Order statistics are monotone in each argument, so the m-th smallest
projection at any s in [a, b] lies in [lo_(m), hi_(m)] (sorted separately),
and the narrowest window of h projections is at least
    LB = max(0, min over a' of lo_(a'+h-1) - hi_(a')).
At a single slope (a = b) LB equals w(s) (Sec. 3.1: the slab height).
"""
from __future__ import annotations

from fractions import Fraction


def lower_bound(xs, ys, h, a: Fraction, b: Fraction) -> Fraction:
    lo, hi = [], []
    for x, y in zip(xs, ys):
        za, zb = Fraction(y) - a * x, Fraction(y) - b * x
        lo.append(min(za, zb))
        hi.append(max(za, zb))
    lo.sort()
    hi.sort()
    n = len(lo)
    m = min(lo[k + h - 1] - hi[k] for k in range(n - h + 1))
    return max(Fraction(0), m)


def width_at(xs, ys, h, s: Fraction) -> Fraction:
    z = sorted(Fraction(y) - s * x for x, y in zip(xs, ys))
    return min(z[k + h - 1] - z[k] for k in range(len(z) - h + 1))


def span_lower_bound(xs, h) -> int:
    """dh: at most m points share one integer x (m the largest multiplicity),
    so any h points take at least ceil(h / m) distinct x values and span at
    least ceil(h / m) - 1 in x."""
    m = max(xs.count(v) for v in set(xs))
    return -(-h // m) - 1


def steep_lower_bound(xs, ys, h, s_abs_min: Fraction) -> Fraction:
    """Lower bound of w(s) for every slope with |s| >= s_abs_min: the h points
    of any window span at least dh in x and at most the y range in y, so their
    projections y - s x spread over at least |s| dh - (max y - min y)."""
    v = s_abs_min * span_lower_bound(list(xs), h) - (max(ys) - min(ys))
    return max(Fraction(0), Fraction(v))
