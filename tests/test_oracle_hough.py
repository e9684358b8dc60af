"""Hough oracle pins: every edge pixel casts exactly one vote per theta
(totals = edges x n_theta); a synthetic image holding one straight line
peaks at that line's (theta, rho) bin; the greedy peak rule never returns two
peaks within the suppression window, takes equal votes in (theta, rho)
order and suppresses a bin exactly on the window's edge; out-of-range rho
clamps to the end bins; a horizontal row gathers untransposed."""
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


def test_peaks_tie_order_and_window_edges():
    # equal votes: smaller theta first, then smaller rho; a bin exactly nms
    # away in both directions is suppressed, one bin further is not
    acc = np.zeros((16, 40), np.int64)
    acc[3, 12] = acc[3, 30] = acc[6, 20] = 9
    acc[8, 22] = 8      # dt = 2, dr = 2 from (6, 20): on the window's edge, suppressed
    acc[9, 20] = 8      # dt = 3 from (6, 20): kept
    acc[6, 23] = 7      # dr = 3 from (6, 20): kept
    pk = hough.peaks(acc, 10, 2, 2)
    assert [(t, r) for t, r, _ in pk][:5] == [(3, 12), (3, 30), (6, 20), (9, 20), (6, 23)]
    assert (8, 22) not in {(t, r) for t, r, _ in pk}
    # top_k ends the list; zero-vote bins (raster order) fill it after the voted ones
    assert [(t, r) for t, r, _ in hough.peaks(acc, 2, 2, 2)] == [(3, 12), (3, 30)]
    assert [v for _, _, v in pk][5:] == [0] * 5


def test_vote_clamp_and_horizontal_gather():
    H = W = 64
    img = np.zeros((H, W), np.uint8)
    img[10, 5:60] = 1                        # the row y = 10 - H/2 = -22, x = -27 .. 27
    n_theta = 8
    cs = hough.tables(n_theta)
    # theta = 0: cos = 1 and sin = 0 exactly, rho = x, bin floor(x + 4)
    # clamped to [0, 8): x <= -4 clamps low (24 pixels), x >= 3 high (25)
    acc = hough.vote(img, n_theta, 8, cs)
    assert acc.sum() == int(img.sum()) * n_theta
    assert acc[0].tolist() == [24, 1, 1, 1, 1, 1, 1, 25]
    # theta = pi/2 (t = n_theta / 2) holds the whole row in the bin of
    # rho = -22; its band gathers exactly the row, not transposed (|sin| > |cos|)
    n_rho = 2 * 91
    acc = hough.vote(img, n_theta, n_rho, cs)
    t = n_theta // 2
    assert acc[t, -22 + n_rho // 2] == int(img.sum())
    x, y, tr = hough.gather(img, (t, -22 + n_rho // 2, int(img.sum())), n_rho, cs, 1.0)
    assert not tr
    assert np.all(y == -22) and x.tolist() == list(range(5 - 32, 60 - 32))
