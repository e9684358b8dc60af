"""Hough + LMS line detection on the GPU against the CPU oracle: vote
accumulators and peaks bit for bit, band sets and their exact LMS fits."""
import ctypes

import numpy as np
import pytest

from oracle import hough as ohough
from paper_1510_01041_gb300 import datagen
from subsample_rule import subsample_mask

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_01041_gb300 import build, lms
    build.build()
    return lms


def run(L, imgs, n_theta, n_rho, top_k, band, nms, max_points=0, seed=0, own_table=False):
    """own_table: the library computes its (cos, sin) table itself (the path
    every caller without a table takes); the oracle always uses its own."""
    cs = ohough.tables(n_theta)
    acc = torch.zeros((imgs.shape[0], n_theta, n_rho), dtype=torch.int32, device="cuda")
    lines = L.hough_refine(torch.from_numpy(imgs).cuda(), n_theta, n_rho, top_k, band, nms, nms,
                           cos_sin=None if own_table else torch.from_numpy(cs).cuda(), acc_out=acc,
                           max_points=max_points, sample_seed=seed)
    return cs, acc.cpu().numpy(), lines


def ols(x, y):
    """Least squares from exact integer sums (one division for the slope)."""
    x = [int(v) for v in x]
    y = [int(v) for v in y]
    n, sx, sy = len(x), sum(x), sum(y)
    sxx, sxy = sum(v * v for v in x), sum(a * b for a, b in zip(x, y))
    den = n * sxx - sx * sx
    if den == 0:
        return None, None
    t1 = (n * sxy - sx * sy) / den
    return t1, (sy - t1 * sx) / n


def compare(orc, L, imgs, cs, acc, lines, n_theta, n_rho, top_k, band, nms, check_sets=None, max_points=0, seed=0):
    for b in range(imgs.shape[0]):
        oacc = ohough.vote(imgs[b], n_theta, n_rho, cs)
        assert np.array_equal(acc[b], oacc), b
        opk = ohough.peaks(oacc, top_k, nms, nms)
        got = [(ln["theta_index"], ln["rho_index"], ln["votes"]) for ln in lines[b * top_k:(b + 1) * top_k]]
        assert got[:len(opk)] == opk
        for k, pk in enumerate(opk):
            if check_sets is not None and k not in check_sets:
                continue
            x, y, tr = ohough.gather(imgs[b], pk, n_rho, cs, band)
            ln = lines[b * top_k + k]
            assert ln["npoints"] == x.size and ln["transposed"] == int(tr)
            if x.size >= 2:
                keep = subsample_mask(seed, b * top_k + k, x.size, max_points)
                x, y = x[keep], y[keep]
                assert ln["nfit"] == x.size, (b, k)
                t1, t2 = ols(x, y)
                if t1 is None:
                    assert np.isnan(ln["ols_theta1"])
                else:
                    assert ln["ols_theta1"] == t1, (b, k)
                    assert abs(ln["ols_theta2"] - t2) <= 1e-12 * max(1.0, abs(t2)), (b, k)
                o = orc.lms_i16(x, y, 0, "sweep")
                f = ln["fit"]
                assert (f["status"], f["w_num"], f["s_num"], f["s_den"], f["t_num"], f["i"], f["j"], f["med_sq"]) == \
                       (o.status, o.w_num, o.s_num, o.s_den, o.t_num, o.i, o.j, o.med_sq), (b, k)


def test_hough_small_images(L, orc):
    imgs = datagen.edge_images(2, 21, height=384, width=512, segments=5, len_min=80, len_max=300, salt=0.01)
    n_theta, n_rho, top_k, band, nms = 180, 2 * int(np.ceil(np.hypot(192, 256))) + 2, 8, 4.0, 5
    cs, acc, lines = run(L, imgs, n_theta, n_rho, top_k, band, nms)
    compare(orc, L, imgs, cs, acc, lines, n_theta, n_rho, top_k, band, nms)


def test_hough_library_table(L, orc):
    """No table passed: the library's own host-computed (cos, sin) table gives
    the oracle's votes, peaks, bands and fits, at the full 1024-angle
    resolution and at an odd one."""
    imgs = datagen.edge_images(2, 22, height=384, width=512, segments=5, len_min=80, len_max=300, salt=0.01)
    n_rho = 2 * int(np.ceil(np.hypot(192, 256))) + 2
    for n_theta in (1024, 331):
        cs, acc, lines = run(L, imgs, n_theta, n_rho, 8, 4.0, 5, own_table=True)
        compare(orc, L, imgs, cs, acc, lines, n_theta, n_rho, 8, 4.0, 5)


def test_hough_full_size_image(L, orc):
    """One image at the full 2048x2048 / 1024 x 2896 configuration; LMS of
    four of its 32 sets checked one by one."""
    imgs = datagen.edge_images(1, 4, height=2048, width=2048)
    cs, acc, lines = run(L, imgs, 1024, 2896, 32, 4.0, 5)
    compare(orc, L, imgs, cs, acc, lines, 1024, 2896, 32, 4.0, 5, check_sets={0, 1, 7, 31})


def test_hough_subsampled_sets(L, orc):
    """Bands subsampled to about 40 points: the kept points follow the
    documented rule (reproduced here from SplitMix64's definition) and their
    exact LMS and least-squares lines match the oracle's."""
    imgs = datagen.edge_images(2, 33, height=384, width=512, segments=5, len_min=150, len_max=300, salt=0.01)
    n_theta, n_rho, top_k, band, nms = 180, 2 * int(np.ceil(np.hypot(192, 256))) + 2, 6, 4.0, 5
    cs, acc, lines = run(L, imgs, n_theta, n_rho, top_k, band, nms, max_points=40, seed=12345)
    assert any(ln["npoints"] > 40 for ln in lines)
    compare(orc, L, imgs, cs, acc, lines, n_theta, n_rho, top_k, band, nms, max_points=40, seed=12345)
