"""O3: exhaustive LMS on tiny inputs, in exact rationals (pure Python).

TEST INFRASTRUCTURE ONLY.  Independent of the sorted-window formulation used
by the C oracle and the CUDA path: it enumerates point subsets instead.

* ``lms_subsets``  -- min over candidate slopes s (all pairwise slopes with
  dx != 0, Sec. 3.3) and over every h-subset T of the range of the
  projections z_k = y_k - s x_k, k in T.  The lexicographic minimum of
  (range, s, centre) and the smallest index pair with that slope.
* ``lms_chebyshev`` -- min over h-subsets T of T's minimax (L-infinity) line
  fit, computed from T's own pairwise slopes only; its value is half the
  LMS slab height (Sec. 3.1: half the points inside a slab of height 2 sqrt(d)).
* ``lms_equioscillation`` -- min over point triples x_a < x_b < x_c of the
  h-th smallest |residual| of the line that equioscillates with respect to
  the triple (Sec. 3.3, Steele & Steiger): slope of (a, c), placed halfway
  between that chord and b.
* ``window_width_at`` -- w(s) for any rational s by subsets (continuous check).
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations


def candidate_slopes(pts):
    s = set()
    for (xa, ya), (xb, yb) in combinations(pts, 2):
        if xa != xb:
            s.add(Fraction(yb - ya, xb - xa))
    return sorted(s)


def window_width_at(pts, h, s):
    """(min range over h-subsets, smallest centre among the minimisers) at slope s."""
    z = [Fraction(y) - s * x for x, y in pts]
    best = None
    for T in combinations(range(len(pts)), h):
        zt = [z[k] for k in T]
        w = max(zt) - min(zt)
        c = (max(zt) + min(zt)) / 2
        if best is None or (w, c) < best:
            best = (w, c)
    return best


def lms_subsets(pts, h=None):
    """Returns (w, theta1, theta2, (i, j)) as Fractions, or None if no slope."""
    n = len(pts)
    if h is None:
        h = n // 2 + 1
    best = None
    for s in candidate_slopes(pts):
        w, c = window_width_at(pts, h, s)
        if best is None or (w, s, c) < best:
            best = (w, s, c)
    if best is None:
        return None
    w, s, c = best
    pair = None
    for i in range(n):
        for j in range(i + 1, n):
            (xa, ya), (xb, yb) = pts[i], pts[j]
            if xa != xb and Fraction(yb - ya, xb - xa) == s:
                pair = (i, j)
                break
        if pair:
            break
    return w, s, c, pair


def chebyshev_value(sub):
    """Minimax residual of the best line through ``sub`` (half its narrowest range)."""
    slopes = candidate_slopes(sub)
    if not slopes:
        ys = [y for _, y in sub]
        return Fraction(max(ys) - min(ys), 2)
    best = None
    for s in slopes:
        z = [Fraction(y) - s * x for x, y in sub]
        r = (max(z) - min(z)) / 2
        best = r if best is None or r < best else best
    return best


def lms_chebyshev(pts, h=None):
    n = len(pts)
    if h is None:
        h = n // 2 + 1
    return min(chebyshev_value([pts[k] for k in T]) for T in combinations(range(n), h))


def lms_equioscillation(pts, h=None):
    """min over triples with distinct x of the h-th smallest |residual| of the
    triple's equioscillating line; None if no such triple."""
    n = len(pts)
    if h is None:
        h = n // 2 + 1
    best = None
    for tri in combinations(range(n), 3):
        a, b, c = sorted(tri, key=lambda k: pts[k][0])
        (xa, ya), (xb, yb), (xc, yc) = pts[a], pts[b], pts[c]
        if not (xa < xb < xc):
            continue
        s = Fraction(yc - ya, xc - xa)
        t2 = ((ya - s * xa) + (yb - s * xb)) / 2
        res = sorted(abs(y - s * x - t2) for x, y in pts)
        v = res[h - 1]
        best = v if best is None or v < best else best
    return best
