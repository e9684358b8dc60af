"""Host restatement of the band subsampling rule of ``lms_hough_refine``
(Sec. 5: random subsampling of a line's supporting points before the LMS).

Point u (raster rank) of fitted set k is kept when the upper 32 bits of
SplitMix64's output function applied to seed ^ ((k << 32 | u) * G), with G
the generator's golden-ratio increment 0x9E3779B97F4A7C15, lie below
floor(max_points * 2^32 / count) (at least 1); a sample of fewer than two
points keeps the whole set.  SplitMix64 is Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014.
"""
import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix_out(z):
    """SplitMix64's output function (the mix applied to each state)."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix_sequence(seed, count):
    """The generator itself: the state advances by GOLDEN, each output is the
    mix of the new state."""
    out, s = [], seed & M64
    for _ in range(count):
        s = (s + GOLDEN) & M64
        out.append(splitmix_out(s))
    return out


def subsample_mask(seed, k, count, max_points):
    """Which band points the sampling rule keeps (raster ranks)."""
    if max_points == 0 or count <= max_points:
        return np.ones(count, bool)
    thr = ((max_points << 32) // count) or 1
    m = np.array([(splitmix_out(seed ^ ((((k << 32) | u) * GOLDEN) & M64)) >> 32) < thr
                  for u in range(count)])
    return m if m.sum() >= 2 else np.ones(count, bool)
