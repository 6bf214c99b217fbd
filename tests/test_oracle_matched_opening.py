"""Pins of the opening with the paper-literal structuring element (erosion
dt2 >= R^2, dilation by the ball |d|^2 <= R^2 for integer R; Section 2.4.1
with the integer radius of Section 2.1, footnote 1): the plain ball-stamping
form against the thresholded-EDT form, against a SciPy restatement of the
three steps, and the shared-bound case against the original opening."""
import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

ndi = pytest.importorskip("scipy.ndimage")

FACE_SLICES = {0: (0, slice(None), slice(None)), 1: (-1, slice(None), slice(None)),
               2: (slice(None), 0, slice(None)), 3: (slice(None), -1, slice(None)),
               4: (slice(None), slice(None), 0), 5: (slice(None), slice(None), -1)}


def scipy_opening(img, d, Te, Td, inlet):
    """Erode by threshold, keep the 6-connected components touching the
    inlet face, dilate with a ball structuring element |d|^2 < Td; the first
    level that reaches a pore voxel is its level."""
    level = np.where(img > 0, -1, 0).astype(np.int32)
    six = ndi.generate_binary_structure(3, 1)
    for i, (te, td) in enumerate(zip(Te, Td)):
        E = (img > 0) & (d >= te)
        lab, _ = ndi.label(E, structure=six)
        ids = np.unique(lab[FACE_SLICES[inlet]])
        keep = np.isin(lab, ids[ids > 0])
        r = int(np.floor(np.sqrt(td - 1)))
        o = np.arange(-r, r + 1)
        ball = (o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2) < td
        D = ndi.binary_dilation(keep, structure=ball) if keep.any() else keep
        level[D & (level == -1)] = i + 1
    return level


@pytest.mark.parametrize("seed", range(10))
def test_plain_edt_and_scipy_agree(seed):
    rng = np.random.default_rng(500 + seed)
    shape = tuple(int(x) for x in rng.integers(6, 16, 3))
    img = S.blobs(shape, 1.5, rng.uniform(0.55, 0.8), rng) if seed % 2 else S.random_image(shape, 0.8, rng)
    d = O.edt(img)
    Te, Td = S.integer_radius_levels(int(d[img > 0].max()) if img.any() else 1)
    inlet = seed % 6
    lp, cp = O.morph_drainage(img, d, Te, inlet=inlet, method="plain", dilate_levels=Td)
    le, ce = O.morph_drainage(img, d, Te, inlet=inlet, method="edt", dilate_levels=Td)
    assert np.array_equal(lp, le) and np.array_equal(cp, ce)
    assert np.array_equal(lp, scipy_opening(img, d, Te, Td, inlet))
    # same bounds: the original opening
    lo, co = O.morph_drainage(img, d, Te, inlet=inlet, method="plain")
    assert np.array_equal(lo, scipy_opening(img, d, Te, Te, inlet))


def test_integer_radius_levels():
    Te, Td = S.integer_radius_levels(50)   # R = 7 .. 1
    assert Te == [49, 36, 25, 16, 9, 4, 1] and Td == [50, 37, 26, 17, 10, 5, 2]
    assert S.integer_radius_levels(1) == ([1], [2])


def test_closed_ball_reaches_the_sphere_surface():
    """A pore cavity |v - c|^2 <= R^2 cut by the inlet face through its
    centre: the centre has dt2 = R^2 + 1 (the nearest solid lies just outside
    the closed ball), so level R erodes to the voxels with dt2 >= R^2 and the
    ball |d|^2 <= R^2 around the centre alone covers the whole cavity, while
    the open ball |d|^2 < R^2 misses its surface shell."""
    R = 4
    n = 2 * R + 3
    x, y, z = np.meshgrid(np.arange(R + 2), np.arange(n), np.arange(n), indexing="ij")
    c = n // 2
    img = ((x ** 2 + (y - c) ** 2 + (z - c) ** 2) <= R * R).astype(np.uint8)
    d = O.edt(img)
    assert d[0, c, c] == R * R + 1
    lc, cc = O.morph_drainage(img, d, [R * R], inlet=0, dilate_levels=[R * R + 1])
    lo, co = O.morph_drainage(img, d, [R * R], inlet=0)
    assert cc[0] == np.count_nonzero(img)
    shell = (x ** 2 + (y - c) ** 2 + (z - c) ** 2) == R * R
    assert co[0] < cc[0] and (lc[shell] == 1).all()
