"""Pins of the host restatement of the band subsampling rule: the generator
against published outputs of SplitMix64's reference implementation, and the
rule's sampling rate and degenerate cases."""
import numpy as np

from subsample_rule import splitmix_sequence, subsample_mask


def test_splitmix_reference_outputs():
    # first outputs of the reference splitmix64.c (Vigna), seeds 1234567 and
    # 1477776061723855037, as published with it and in its ports' test suites
    assert splitmix_sequence(1234567, 5) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert splitmix_sequence(1477776061723855037, 3) == [
        1985237415132408290, 2979275885539914483, 13511426838097143398]


def test_subsample_rate_and_edges():
    # kept fraction close to max_points / count over many sets (binomial)
    count, mp = 1000, 128
    kept = [subsample_mask(7, k, count, mp).sum() for k in range(40)]
    mean = float(np.mean(kept))
    assert abs(mean - mp) < 4 * np.sqrt(mp * (1 - mp / count) / len(kept)) + 1
    # different sets and seeds draw different samples
    assert not np.array_equal(subsample_mask(7, 0, count, mp), subsample_mask(7, 1, count, mp))
    assert not np.array_equal(subsample_mask(7, 0, count, mp), subsample_mask(8, 0, count, mp))
    # max_points 0 or a set no larger than max_points keeps everything
    assert subsample_mask(3, 0, 50, 0).all()
    assert subsample_mask(3, 0, 50, 50).all()
    # max_points = 1 of 4096 draws about one point: a draw of fewer than two
    # keeps the whole set, a draw of two or more is kept as drawn
    sums = [int(subsample_mask(3, k, 4096, 1).sum()) for k in range(24)]
    assert 4096 in sums
    assert all(s == 4096 or 2 <= s < 16 for s in sums)
    assert any(2 <= s < 16 for s in sums)
