"""Pins of the drainage envelope (Section 2.2.2 and Section 3.1.1: the
envelope of the invasion's peak pressures against the opening's curve), by
integer counts: the invasion's invaded count at the step before its
running-minimum sphere size first drops below an opening level."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S


def test_hand_example():
    # five steps with radii^2 9, 9, 4, 9, 1 invading 2, 1, 3, 1, 2 voxels
    seq = np.array([1, 1, 2, 3, 3, 3, 4, 5, 5, 0, -1], np.int32).reshape(1, 1, 11)
    r2 = np.array([9, 9, 4, 9, 1], np.int32)
    k, n = O.pc_envelope(seq, r2, [10, 9, 5, 4, 2, 1])
    # T=10: step 1 already below -> 0 steps; T=9: steps 1-2; T=5, 4: steps 1-4
    # (step 4 has r2 = 9 but comes after the drop to 4 only for T > 4);
    # T=2: steps 1-4; T=1: all five
    assert list(k) == [0, 2, 2, 4, 4, 5]
    assert list(n) == [0, 3, 3, 7, 7, 9]


def test_tube_closed_form():
    """Straight tube of radius R: the first ceil(nx/R) steps are the axis
    spheres (r2 = R^2), so at the opening level R^2 the invasion holds the
    union of those balls (computed here from the geometry), while the
    opening at R^2 holds the whole tube (its axis erodes to dt2 = R^2 and the
    ball d^2 < R^2 around the axis is the tube)."""
    R, nx = 8, 50
    img = S.tube(nx, R)
    d = O.edt(img)
    seq, r2, cen, st, K = O.invade(img, d, inlet=0)
    k, n = O.pc_envelope(seq, r2, [R * R])
    nb = math.ceil(nx / R)
    assert k[0] == nb
    c = img.shape[1] // 2
    x, y, z = np.meshgrid(np.arange(nx), np.arange(img.shape[1]), np.arange(img.shape[2]), indexing="ij")
    covered = np.zeros(img.shape, bool)
    for j in range(nb):
        covered |= (x - j * R) ** 2 + (y - c) ** 2 + (z - c) ** 2 < R * R
    assert n[0] == int(np.count_nonzero(covered & (img > 0)))
    lev, cnt = O.morph_drainage(img, d, [R * R], inlet=0)
    assert cnt[0] == int(np.count_nonzero(img))
    assert n[0] < cnt[0]   # R = 8 leaves crevices between the axis spheres for later steps


@pytest.mark.parametrize("seed", range(5))
def test_monotone_and_bounded(seed):
    rng = np.random.default_rng(300 + seed)
    img = S.blobs((18, 20, 16), 2.0, 0.6, rng) if seed % 2 else S.sphere_pack((20, 18, 22), 3, 0.45, rng)
    d = O.edt(img)
    seq, r2, cen, st, K = O.invade(img, d, inlet=seed % 6)
    T = S.mio_levels(int(d[img > 0].max()), 16)
    k, n = O.pc_envelope(seq, r2, T)
    assert (np.diff(k) >= 0).all() and (np.diff(n) >= 0).all()
    # every step before kstar has r2 >= T, and step kstar + 1 (if any) is below
    for T_i, k_i in zip(T, k):
        assert (r2[:k_i] >= T_i).all()
        assert k_i == K or r2[k_i] < T_i
    assert n[-1] <= np.count_nonzero(seq >= 1)
    k1, n1 = O.pc_envelope(seq, r2, [1])
    assert k1[0] == K and n1[0] == np.count_nonzero(seq >= 1)
