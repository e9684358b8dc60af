"""Hough oracle pins: every edge pixel casts exactly one vote per theta
(totals = edges x n_theta); a synthetic image holding one straight line
peaks at that line's (theta, rho) bin; the greedy peak rule never returns two
peaks within the suppression window."""
import numpy as np

from oracle import hough


def test_vote_totals_and_line_peak():
    H = W = 128
    img = np.zeros((H, W), np.uint8)
    # the vertical line x = 20 (theta = 0, rho = 20 - W/2 = -44)
    img[:, 20] = 1
    rng = np.random.default_rng(0)
    img[rng.integers(0, H, 40), rng.integers(0, W, 40)] = 1
    n_theta, n_rho = 64, 182
    cs = hough.tables(n_theta)
    acc = hough.vote(img, n_theta, n_rho, cs)
    assert acc.sum() == int(img.sum()) * n_theta
    pk = hough.peaks(acc, 3, 2, 2)
    assert pk[0][0] == 0 and pk[0][1] == -44 + n_rho // 2 and pk[0][2] >= H
    for a in range(len(pk)):
        for b in range(a):
            assert not (abs(pk[a][0] - pk[b][0]) <= 2 and abs(pk[a][1] - pk[b][1]) <= 2)
    x, y, tr = hough.gather(img, pk[0], n_rho, cs, 1.0)
    assert tr  # theta = 0 is a vertical line: fitted in the swapped frame
    assert np.all(y == -44)
