"""Pins of the post-processing outputs of Sections 2.2.2-2.2.3: the
sphere-size image and re-ranked trapping with the surviving steps' radii."""
import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S


@pytest.mark.parametrize("seed", range(6))
def test_size_image_lies_inside_each_steps_ball(seed):
    rng = np.random.default_rng(seed)
    img = S.sphere_pack((18, 16, 20), 3, 0.45, rng)
    d = O.edt(img)
    seq, r2, cen, st, K = O.invade(img, d, inlet=seed % 6)
    size = O.size_image(seq, r2)
    assert (size[img == 0] == 0).all() and (size[(img > 0) & (seq == -1)] == -1).all()
    v = np.argwhere(seq >= 1)
    c = np.stack(np.unravel_index(cen[seq[seq >= 1] - 1], img.shape), 1)
    assert (((v - c) ** 2).sum(1) < size[seq >= 1]).all()
    assert (size[seq >= 1] == d.ravel()[cen[seq[seq >= 1] - 1]]).all()


def test_size_image_tube():
    R = 5
    img = S.tube(40, R)
    seq, r2, cen, st, K = O.invade(img, O.edt(img), inlet=0)
    size = O.size_image(seq, r2)
    cy, cz = img.shape[1] // 2, img.shape[2] // 2
    assert (size[:, cy, cz] == R * R).all()


@pytest.mark.parametrize("seed", range(6))
def test_rerank_radii(seed):
    rng = np.random.default_rng(50 + seed)
    img = S.blobs((20, 18, 22), 2.0, 0.6, rng)
    d = O.edt(img)
    seq, r2, cen, st, K = O.invade(img, d, inlet=0)
    tr, so_nr = O.trapping(seq, 1, rerank=False)
    tr2, so, r2o = O.rerank_radii(seq, r2, 1)
    kept = np.unique(so_nr[so_nr >= 1])
    assert np.array_equal(tr, tr2) and len(r2o) == len(kept)
    # dense renumbering in the old order
    assert np.array_equal(so[so >= 1], np.searchsorted(kept, so_nr[so_nr >= 1]) + 1)
    assert np.array_equal(so < 1, so_nr < 1)
    # the re-ranked curve is the original one restricted to surviving steps
    S1, P1 = O.pc_curve(so_nr, r2)[:2]
    S2, P2 = O.pc_curve(so, r2o)[:2]
    assert np.array_equal(P2, P1[kept - 1]) and np.array_equal(S2, S1[kept - 1])
