"""Pins of the equal-saturation comparison (Section 3.1.1, by integer
counts) between an invasion sequence and opening levels."""
import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S


def test_hand_example():
    # a chain of six pore voxels invaded in order; opening levels by hand
    seq = np.array([1, 2, 3, 4, 5, 6], np.int32).reshape(1, 1, 6)
    level = np.array([1, 1, 2, -1, 2, 3], np.int32).reshape(1, 1, 6)
    k, diff, n = O.equal_saturation(seq, level, 3)
    # level 0: {0,1} vs steps <= 2 -> same; level 1: {0,1,2,4} vs steps <= 4
    # -> {3} and {4} differ; level 2: {0,1,2,4,5} vs steps <= 5 -> {3}, {5}
    assert list(n) == [2, 4, 5] and list(k) == [2, 4, 5] and list(diff) == [0, 2, 2]


def test_unreachable_count_takes_the_last_step():
    seq = np.array([0, 1, 2, -1], np.int32).reshape(1, 1, 4)
    level = np.array([0, 1, 1, 1], np.int32).reshape(1, 1, 4)
    k, diff, n = O.equal_saturation(seq, level, 1)
    assert list(n) == [3] and list(k) == [2] and list(diff) == [1]


@pytest.mark.parametrize("seed", range(6))
def test_levels_cut_from_the_sequence_agree_exactly(seed):
    """Opening levels made by cutting the invasion's own sequence at chosen
    steps have zero difference at every level (every step invades at least
    its centre, so the matched step is the cut itself)."""
    rng = np.random.default_rng(seed)
    img = S.blobs((16, 14, 18), 2.0, 0.6, rng)
    seq, r2, cen, st, K = O.invade(img, O.edt(img), inlet=seed % 6)
    cuts = np.unique(rng.integers(1, max(K, 2), 5))
    level = np.where(img > 0, -1, 0).astype(np.int32)
    for i, c in reversed(list(enumerate(cuts))):
        level[(seq >= 1) & (seq <= c)] = i + 1
    k, diff, n = O.equal_saturation(seq, level, len(cuts))
    assert list(k) == list(cuts) and (diff == 0).all()


@pytest.mark.parametrize("seed", range(4))
def test_difference_bounds(seed):
    rng = np.random.default_rng(40 + seed)
    img = S.blobs((20, 20, 20), 2.0, 0.6, rng)
    d = O.edt(img)
    seq = O.invade(img, d, inlet=0)[0]
    T = S.mio_levels(int(d[img > 0].max()), 12)
    level = O.morph_drainage(img, d, T, inlet=0)[0]
    k, diff, n = O.equal_saturation(seq, level, len(T))
    cum = np.array([np.count_nonzero((seq >= 1) & (seq <= kk)) for kk in k])
    assert (np.diff(k) >= 0).all() and (np.diff(n) >= 0).all()
    assert (diff >= np.abs(n - cum)).all() and ((diff - n - cum) % 2 == 0).all()
    assert (diff <= n + cum).all()
