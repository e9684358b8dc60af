"""The seeded input generators (no GPU): the counter-based SplitMix64 stream
reproduces the generator's published reference outputs, and the synthetic
line images hold what their documentation states."""
import math

import numpy as np

from paper_1510_01041_gb300 import datagen


def test_splitmix64_reference_outputs():
    # SplitMix64 (Steele, Lea and Flood 2014) from state 0: the first three
    # outputs of the published reference generator
    got = [int(v) for v in datagen.Stream(0).u64(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_single_line_images_geometry():
    imgs, truth = datagen.single_line_images(6, 3, size=512, noise=0.0, keep=1.0, len_min=200, len_max=300)
    h = 256
    for b in range(6):
        s, c = truth[b]
        assert 0.25 - 1e-12 <= abs(s) <= 4.0 + 1e-12
        rows, cols = np.nonzero(imgs[b])
        x, y = cols - h, rows - h
        assert x.size >= 200
        # every pixel is the rounding of the true line along its major axis
        if abs(s) <= 1:
            assert np.all(np.abs(y - (s * x + c)) <= 0.5 + 1e-9)
        else:
            assert np.all(np.abs(x - (y - c) / s) <= 0.5 + 1e-9)


def test_single_line_images_noise_and_keep_rate():
    imgs, _ = datagen.single_line_images(4, 8, size=512, noise=0.004, keep=0.5, len_min=400, len_max=400)
    total = imgs.reshape(4, -1).sum(axis=1).astype(np.int64)
    # 400 line pixels kept with p = 0.5 plus ~0.004 * 512^2 = 1049 noise pixels
    assert np.all(np.abs(total - (200 + 1049)) < 5 * math.sqrt(200 + 1049))
    same, _ = datagen.single_line_images(4, 8, size=512, noise=0.004, keep=0.5, len_min=400, len_max=400)
    assert np.array_equal(imgs, same)               # a pure function of the seed
