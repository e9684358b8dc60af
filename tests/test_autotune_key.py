"""The autotuner's cache key depends on the device and the mix of set sizes
only: the order of the sets does not change it, a different size mix (also
within one power of two) or device does."""
import numpy as np

from paper_1510_01041_gb300 import autotune


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)])


def test_key_ignores_set_order_and_separates_mixes():
    rng = np.random.default_rng(0)
    sizes = rng.integers(64, 4096, 200)
    k = autotune._key(_offsets(sizes), "GPU-A")
    assert k == autotune._key(_offsets(rng.permutation(sizes)), "GPU-A")
    assert k != autotune._key(_offsets(sizes), "GPU-B")
    assert k != autotune._key(_offsets(np.full(200, 64)), "GPU-A")
    assert k != autotune._key(_offsets(sizes[:150]), "GPU-A")   # set count is part of the key


def test_key_separates_sizes_within_one_octave():
    # all sets at 1100 points and all at 2000 fall in one power-of-two bin
    assert autotune._key(_offsets(np.full(300, 1100)), "G") != autotune._key(_offsets(np.full(300, 2000)), "G")
    assert autotune._key(_offsets(np.full(300, 1100)), "G") != autotune._key(_offsets(np.full(300, 1101)), "G")
