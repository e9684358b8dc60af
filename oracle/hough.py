"""CPU oracle of Hough voting, peak selection and band gathering (Sec. 5).

TEST INFRASTRUCTURE ONLY (numpy float32, independent of the CUDA kernels).
Conventions, chosen where the paper is silent: image-centre coordinates
(x - W/2, y - H/2); theta_t = pi t / n_theta; rho bin
floor(x cos_t + y sin_t + n_rho/2) clamped to [0, n_rho), with the two
products and the sum each rounded to float32 (numpy float32 arithmetic does
exactly that); peaks greedily in the order (votes desc, t asc, rho asc),
skipping bins within +-nms_theta / +-nms_rho of a taken peak; a peak's band
holds the edge pixels with |x cos + y sin - rho_c| <= band, rho_c the bin
centre (rho index - n_rho/2 + 0.5), in raster order; near-vertical peaks
(|sin| < |cos|) swap x and y.
"""
from __future__ import annotations

import numpy as np


def tables(n_theta: int) -> np.ndarray:
    """(cos, sin) float32 pairs, shape [n_theta, 2]."""
    th = np.pi * np.arange(n_theta, dtype=np.float64) / n_theta
    return np.stack([np.cos(th), np.sin(th)], axis=1).astype(np.float32)


def edge_points(img):
    H, W = img.shape
    yy, xx = np.nonzero(img)                      # raster order
    return (xx - W // 2).astype(np.int64), (yy - H // 2).astype(np.int64)


def vote(img, n_theta, n_rho, cs):
    xc, yc = edge_points(img)
    xf, yf = xc.astype(np.float32), yc.astype(np.float32)
    half = np.float32(n_rho // 2)
    acc = np.zeros((n_theta, n_rho), dtype=np.int64)
    for t in range(n_theta):
        rho = (xf * cs[t, 0]) + (yf * cs[t, 1])
        r = np.floor(rho + half).astype(np.int64)
        r = np.clip(r, 0, n_rho - 1)
        acc[t] = np.bincount(r, minlength=n_rho)
    return acc


def peaks(acc, top_k, nms_t, nms_r):
    n_theta, n_rho = acc.shape
    flat = acc.ravel()
    order = np.lexsort((np.arange(flat.size), -flat))   # votes desc, then (t, r) ascending
    taken = []
    for k in order:
        if len(taken) == top_k:
            break
        v = int(flat[k])
        t, r = divmod(int(k), n_rho)
        if any(abs(t - a) <= nms_t and abs(r - b) <= nms_r for a, b, _ in taken):
            continue
        taken.append((t, r, v))
    return taken


def gather(img, peak, n_rho, cs, band):
    xc, yc = edge_points(img)
    t, r, _ = peak
    c, s = cs[t, 0], cs[t, 1]
    rho = (xc.astype(np.float32) * c) + (yc.astype(np.float32) * s)
    rc = np.float32(r - n_rho // 2) + np.float32(0.5)
    keep = np.abs(rho - rc) <= np.float32(band)
    x, y = xc[keep], yc[keep]
    transposed = bool(abs(s) < abs(c))
    if transposed:
        x, y = y, x
    return x.astype(np.int16), y.astype(np.int16), transposed
