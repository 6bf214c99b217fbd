"""Pins of inlet masks in the oracle invasion (Section 2.1: the inlets are
a Boolean image and may lie inside the image)."""
import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S


def face_mask(shape, face):
    m = np.zeros(shape, np.uint8)
    ax, end = face // 2, face % 2
    idx = [slice(None)] * 3
    idx[ax] = shape[ax] - 1 if end else 0
    m[tuple(idx)] = 1
    return m


@pytest.mark.parametrize("seed", range(12))
def test_face_mask_equals_face(seed):
    rng = np.random.default_rng(seed)
    img = S.random_image(tuple(int(x) for x in rng.integers(2, 12, 3)), rng.uniform(0.4, 0.9), rng)
    d = O.edt(img)
    face = seed % 6
    a = O.invade(img, d, inlet=face)
    b = O.invade(img, d, inlet=3 - face % 3, mask=face_mask(img.shape, face))
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("seed", range(12))
def test_scan_equals_heap_with_random_masks(seed):
    rng = np.random.default_rng(100 + seed)
    img = S.random_image(tuple(int(x) for x in rng.integers(2, 10, 3)), rng.uniform(0.4, 0.9), rng)
    d = O.edt(img)
    mask = (rng.random(img.shape) < rng.uniform(0.005, 0.1)).astype(np.uint8)
    a = O.invade(img, d, mask=mask, method="scan")
    b = O.invade(img, d, mask=mask, method="heap")
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    # invaded voxels are exactly the pore components that hold an inlet voxel
    import scipy.ndimage as nd
    lab, _ = nd.label(img > 0, structure=nd.generate_binary_structure(3, 1))
    seeds = np.unique(lab[(mask > 0) & (img > 0)])
    assert np.array_equal(a[0] >= 1, np.isin(lab, seeds[seeds > 0]))


def test_interior_inlet_at_a_spherical_pore_centre():
    R, n = 6, 17
    z, y, x = np.indices((n, n, n))
    c = n // 2
    img = (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) < R * R).astype(np.uint8)
    d = O.edt(img)
    mask = np.zeros_like(img)
    mask[c, c, c] = 1
    seq, r2, cen, st, K = O.invade(img, d, mask=mask)
    # the centre is the only candidate; its ball d^2 < R^2 is the whole pore
    assert d[c, c, c] == R * R and K == 1 and list(r2) == [R * R]
    assert (seq[img > 0] == 1).all() and (seq[img == 0] == 0).all()


def test_mask_on_solid_only_invades_nothing():
    img = S.random_image((6, 7, 8), 0.6, np.random.default_rng(3))
    mask = (img == 0).astype(np.uint8)
    seq, r2, cen, st, K = O.invade(img, O.edt(img), mask=mask)
    assert K == 0 and (seq[img > 0] == -1).all()
