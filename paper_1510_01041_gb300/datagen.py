"""Seeded synthetic inputs for the exact 2D LMS line estimator.

This module only draws random point sets and edge images.  It contains none
of the estimator's arithmetic, so both the CUDA path and the CPU oracle can
take their inputs from it.

Randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here as a
counter-based stream: the k-th output is mix64(seed + (k + 1) * golden).
Every workload is therefore a pure function of its seed, on any machine.

Workloads (the paper measures on "random point sets" of 128/256/512 points,
Sec. 4 Table 1, and on synthetic edge images, Sec. 5.1; these generators
stand in for them):

* ``line_with_outliers``  -- integer inliers on y = round(0.7 x + 100) plus
  uniform integer noise, and uniform integer outliers.
* ``sloped``              -- same, with a random slope angle and intercept.
* ``gaussian_f32``        -- float32 inliers around a random line, Gaussian
  outliers.
* ``batch``               -- many ``sloped`` instances with log-uniform sizes.
* ``edge_images``         -- binary images with random line segments and salt.
* ``single_line_images``  -- binary images with one line segment whose pixels
  are kept with probability 0.5, plus salt (the synthetic images of the
  paper's line-detection experiments, Sec. 5.1); returns the true lines.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.seed + k * _GOLDEN)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers in [lo, hi) by 32x32 multiply-high (range < 2**32)."""
        span = hi - lo
        assert 0 < span < 2 ** 32
        top = (self.u64(n) >> np.uint64(32)).astype(np.uint64)
        with np.errstate(over="ignore"):
            v = (top * np.uint64(span)) >> np.uint64(32)
        return v.astype(np.int64) + lo

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")


def n_outliers(n: int, frac: float) -> int:
    return min(n, int(math.ceil(frac * n - 1e-9)))


def line_with_outliers(n: int, seed: int, outlier_frac: float = 0.4):
    """Integer points: inliers on round(0.7x + 100) + U{-3..3}, x in [-8192, 8192);
    outliers uniform in [-16384, 16384)^2; shuffled.  Returns int16 (x, y)."""
    st = Stream(seed)
    n_out = n_outliers(n, outlier_frac)
    n_in = n - n_out
    xi = st.integers(-8192, 8192, n_in)
    # round-half-up of 0.7 x + 100 written in integers
    yi = (7 * xi + 1005) // 10 + st.integers(-3, 4, n_in)
    xo = st.integers(-16384, 16384, n_out)
    yo = st.integers(-16384, 16384, n_out)
    x = np.concatenate([xi, xo])
    y = np.concatenate([yi, yo])
    p = st.permutation(n)
    return x[p].astype(np.int16), y[p].astype(np.int16)


def sloped(n: int, seed: int, outlier_frac: float, phi_max: float = 1.5,
           noise: int = 3):
    """Integer points on a random line: angle U(-phi_max, phi_max), intercept
    U{-1000..1000}, inlier noise U{-noise..noise}; the inlier x-range shrinks
    so |y| stays within int16.  Outliers uniform in [-16384, 16384)^2."""
    st = Stream(seed)
    phi = (st.uniform(1)[0] * 2.0 - 1.0) * phi_max
    m = math.tan(phi)
    c = int(st.integers(-1000, 1001, 1)[0])
    n_out = n_outliers(n, outlier_frac)
    n_in = n - n_out
    xr = 8192
    if abs(m) > 1e-12:
        xr = max(16, min(8192, int((16383 - 1000 - noise - 1) / abs(m))))
    xi = st.integers(-xr, xr, n_in)
    yi = np.rint(m * xi.astype(np.float64) + c).astype(np.int64)
    yi += st.integers(-noise, noise + 1, n_in)
    xo = st.integers(-16384, 16384, n_out)
    yo = st.integers(-16384, 16384, n_out)
    x = np.concatenate([xi, xo])
    y = np.clip(np.concatenate([yi, yo]), -32768, 32767)
    p = st.permutation(n)
    return x[p].astype(np.int16), y[p].astype(np.int16), dict(phi=phi, c=c)


def gaussian_f32(n: int, seed: int, outlier_frac: float = 0.4):
    """Float32 points: inliers x ~ N(0, 1000^2), y = tan(phi) x + c + N(0, 2^2)
    with phi ~ U(-1.4, 1.4), c ~ N(0, 100^2); outliers x, y ~ N(0, 1000^2)."""
    st = Stream(seed)
    phi = (st.uniform(1)[0] * 2.0 - 1.0) * 1.4
    c = st.normal(1)[0] * 100.0
    n_out = n_outliers(n, outlier_frac)
    n_in = n - n_out
    xi = st.normal(n_in) * 1000.0
    yi = math.tan(phi) * xi + c + st.normal(n_in) * 2.0
    xo = st.normal(n_out) * 1000.0
    yo = st.normal(n_out) * 1000.0
    x = np.concatenate([xi, xo])
    y = np.concatenate([yi, yo])
    p = st.permutation(n)
    return x[p].astype(np.float32), y[p].astype(np.float32)


def batch(num: int, seed: int, n_min: int = 64, n_max: int = 4096,
          frac_max: float = 0.45, phi_max: float = 1.5):
    """Many ``sloped`` instances: n = floor(n_min * (n_max/n_min)^u), outlier
    fraction U(0, frac_max).  Returns CSR (x, y, offsets[num+1])."""
    st = Stream(seed)
    u = st.uniform(num)
    fr = st.uniform(num) * frac_max
    ratio = n_max / n_min
    sizes = np.minimum(n_max, np.floor(n_min * ratio ** u).astype(np.int64))
    xs, ys = [], []
    for b in range(num):
        x, y, _ = sloped(int(sizes[b]), seed * 1000003 + b + 1, float(fr[b]), phi_max)
        xs.append(x)
        ys.append(y)
    offsets = np.zeros(num + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.concatenate(xs), np.concatenate(ys), offsets


def edge_images(num: int, seed: int, height: int = 2048, width: int = 2048,
                segments: int = 16, len_min: int = 200, len_max: int = 1500,
                salt: float = 0.05):
    """Binary edge images (uint8 0/1, shape [num, height, width]).  Each holds
    ``segments`` random segments of length U[len_min, len_max] px sampled at
    unit steps with integer jitter U{-1,0,1} on both coordinates, plus salt
    pixels set with probability ``salt``."""
    img = np.zeros((num, height, width), dtype=np.uint8)
    for b in range(num):
        st = Stream(seed * 7919 + b + 1)
        for _ in range(segments):
            L = int(st.integers(len_min, len_max + 1, 1)[0])
            ang = st.uniform(1)[0] * math.pi
            cx = st.uniform(1)[0] * width
            cy = st.uniform(1)[0] * height
            t = np.arange(L + 1, dtype=np.float64) - L / 2.0
            px = np.rint(cx + t * math.cos(ang)).astype(np.int64) + st.integers(-1, 2, L + 1)
            py = np.rint(cy + t * math.sin(ang)).astype(np.int64) + st.integers(-1, 2, L + 1)
            ok = (px >= 0) & (px < width) & (py >= 0) & (py < height)
            img[b, py[ok], px[ok]] = 1
        u = st.u64(height * width)
        thresh = np.uint64(int(salt * 2.0 ** 64))
        img[b].reshape(-1)[u < thresh] = 1
    return img


def single_line_images(num: int, seed: int, size: int = 1024, noise: float = 0.001, keep: float = 0.5,
                       len_min: int = 400, len_max: int = 900):
    """Binary images (uint8 0/1, [num, size, size]) each with one straight
    segment: the digital line through a random point of the central half of
    the image at a random angle with |tan| in [0.25, 4], of length
    U[len_min, len_max] px along its major axis, each pixel kept with
    probability ``keep``; plus salt pixels set with probability ``noise``.
    Returns (images, truth) with truth[b] = (slope, intercept) of the
    generating line in image-centre coordinates (x - size/2, y - size/2):
    y = slope x + intercept."""
    img = np.zeros((num, size, size), dtype=np.uint8)
    truth = np.zeros((num, 2), dtype=np.float64)
    h = size // 2
    for b in range(num):
        st = Stream(seed * 104729 + b + 1)
        a = math.atan(0.25) + st.uniform(1)[0] * (math.atan(4.0) - math.atan(0.25))
        if st.uniform(1)[0] < 0.5:
            a = -a
        s = math.tan(a)
        cx = (st.uniform(1)[0] - 0.5) * h
        cy = (st.uniform(1)[0] - 0.5) * h
        c = cy - s * cx
        L = int(st.integers(len_min, len_max + 1, 1)[0])
        t = np.arange(L + 1, dtype=np.float64) - L / 2.0
        if abs(s) <= 1.0:
            x = np.rint(cx + t).astype(np.int64)
            y = np.rint(s * x + c).astype(np.int64)
        else:
            y = np.rint(cy + t).astype(np.int64)
            x = np.rint((y - c) / s).astype(np.int64)
        on = st.uniform(L + 1) < keep
        col, row = x + h, y + h
        ok = on & (col >= 0) & (col < size) & (row >= 0) & (row < size)
        img[b, row[ok], col[ok]] = 1
        u = st.u64(size * size)
        img[b].reshape(-1)[u < np.uint64(int(noise * 2.0 ** 64))] = 1
        truth[b] = (s, c)
    return img, truth
