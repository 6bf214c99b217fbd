"""Pins of the paper-literal invasion oracle (Section 2.1 as printed: cross
dilation of inlets plus past insertion points, every tied maximum at once,
truncated integer radius, dt zeroed at insertion points).

The C oracle's two variants (the definition, rescanning every step, and a
queue) are checked against each other, against an independent set-based
restatement written here with SciPy's binary dilation, against the straight
tube's closed form and against invariants that any correct run satisfies."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

nd = pytest.importorskip("scipy.ndimage")


def face_mask(shape, face):
    m = np.zeros(shape, bool)
    ax, end = face // 2, face % 2
    idx = [slice(None)] * 3
    idx[ax] = shape[ax] - 1 if end else 0
    m[tuple(idx)] = True
    return m


def literal_sets(img, dt2, face):
    """Section 2.1 step by step on whole-image Boolean sets."""
    img = img.astype(bool)
    inlets = face_mask(img.shape, face)
    dt = dt2.astype(np.int64).copy()
    seq = np.where(img, -1, 0).astype(np.int64)
    cstep = np.zeros(img.shape, np.int64)
    cross = nd.generate_binary_structure(3, 1)
    r2s, counts = [], []
    k = 0
    while True:
        cand = nd.binary_dilation(inlets, structure=cross)
        best = int(dt[cand].max()) if cand.any() else 0
        if best == 0:
            break
        k += 1
        pts = np.argwhere(cand & (dt == best))
        R = math.isqrt(best)
        offs = [(a, b, c) for a in range(-R, R + 1) for b in range(-R, R + 1) for c in range(-R, R + 1)
                if a * a + b * b + c * c <= R * R]
        for p in pts:
            for o in offs:
                q = p + o
                if (q < 0).any() or (q >= img.shape).any():
                    continue
                q = tuple(q)
                if img[q] and seq[q] == -1:
                    seq[q] = k
        for p in pts:
            cstep[tuple(p)] = k
            inlets[tuple(p)] = True
            dt[tuple(p)] = 0
        r2s.append(R * R)
        counts.append(len(pts))
    return seq, cstep, np.array(r2s), np.array(counts), k


def check_same(r, ref):
    seq, cstep, r2, cnt, st, K = r
    assert st == 0
    assert K == ref[4]
    assert np.array_equal(seq, ref[0]) and np.array_equal(cstep, ref[1])
    assert np.array_equal(r2, ref[2]) and np.array_equal(cnt, ref[3])


@pytest.mark.parametrize("seed", range(40))
def test_literal_oracle_equals_set_restatement(seed):
    rng = np.random.default_rng(1000 + seed)
    shape = tuple(int(x) for x in rng.integers(1, 8, 3))
    img = S.random_image(shape, rng.uniform(0.3, 0.95), rng)
    d = O.edt(img)
    face = int(rng.integers(0, 6))
    ref = literal_sets(img, d, face)
    check_same(O.invade_literal(img, d, face, method="scan"), ref)
    check_same(O.invade_literal(img, d, face, method="queue"), ref)


@pytest.mark.parametrize("seed", range(8))
def test_literal_queue_equals_scan_on_blobs(seed):
    rng = np.random.default_rng(2000 + seed)
    img = S.blobs((14, 12, 16), rng.uniform(1.0, 2.5), rng.uniform(0.5, 0.8), rng)
    d = O.edt(img)
    face = seed % 6
    a = O.invade_literal(img, d, face, method="scan")
    b = O.invade_literal(img, d, face, method="queue")
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("R", [2, 3, 4, 8])
def test_literal_tube_closed_form(R):
    nx = 6 * R + 5
    img = S.tube(nx, R)
    d = O.edt(img)
    seq, cstep, r2, cnt, st, K = O.invade_literal(img, d, 0)
    cy, cz = img.shape[1] // 2, img.shape[2] // 2
    assert d[0, cy, cz] == R * R
    # step 1: the two axis voxels x = 0 and x = 1 tie; then one axis voxel per step
    assert cnt[0] == 2 and cstep[0, cy, cz] == 1 and cstep[1, cy, cz] == 1
    for x in range(2, nx):
        assert cstep[x, cy, cz] == x
        assert cnt[x - 1] == 1
    assert (r2[: nx - 1] == R * R).all()
    # axis voxel x is first covered by the ball of step max(1, x - R)
    for x in range(nx):
        assert seq[x, cy, cz] == max(1, x - R)
    # breakthrough: the outlet face is reached at step nx - 1 - R with the
    # integer radius R, i.e. Pc = 2 sigma / (R voxel) (theta = 180 deg)
    first = int(seq[nx - 1][seq[nx - 1] > 0].min())
    assert first == nx - 1 - R
    S_, Pc = O.pc_curve(seq, r2)[:2]
    assert Pc[first - 1] == np.float32(2 * 0.072 / (R * 5e-6))


@pytest.mark.parametrize("seed", range(6))
def test_literal_invariants(seed):
    rng = np.random.default_rng(3000 + seed)
    img = S.sphere_pack((20, 18, 22), int(rng.integers(2, 4)), rng.uniform(0.4, 0.6), rng)
    d = O.edt(img)
    face = seed % 6
    seq, cstep, r2, cnt, st, K = O.invade_literal(img, d, face)
    assert st == 0 and K == len(r2) == len(cnt)
    # insertion points of a step share one value, whose truncated root is R
    for k in range(1, K + 1):
        vals = np.unique(d[cstep == k])
        assert len(vals) == 1 and math.isqrt(int(vals[0])) ** 2 == r2[k - 1]
        assert (cstep == k).sum() == cnt[k - 1]
    # the values of successive steps never come from an emptied candidate set
    assert (cnt >= 1).all()
    # every voxel of step k lies in a step-k sphere
    for k in range(1, K + 1):
        pts = np.argwhere(cstep == k)
        vox = np.argwhere(seq == k)
        if len(vox) == 0:
            continue
        dd = ((vox[:, None, :] - pts[None, :, :]) ** 2).sum(-1).min(1)
        assert (dd <= r2[k - 1]).all()
    # only pore is written; insertion points are exactly the pore voxels
    # joined through pore to the inlet face or its face neighbours
    assert (seq[img == 0] == 0).all()
    start = img.astype(bool) & nd.binary_dilation(face_mask(img.shape, face),
                                                  structure=nd.generate_binary_structure(3, 1))
    lab, _ = nd.label(img.astype(bool), structure=nd.generate_binary_structure(3, 1))
    reach = np.isin(lab, np.unique(lab[start])) & (lab > 0)
    assert np.array_equal(cstep > 0, reach)
    # every insertion point is invaded no later than its own step
    assert (seq[cstep > 0] <= cstep[cstep > 0]).all() and (seq[cstep > 0] >= 1).all()


def test_literal_no_solid_and_all_solid():
    img = np.ones((5, 4, 3), np.uint8)
    d = O.edt(img)
    seq, cstep, r2, cnt, st, K = O.invade_literal(img, d, 0)
    # every candidate ties at +infinity: layers x = 0, 1 at step 1, then one layer per step
    assert (seq == 1).all() and K == 4 and list(cnt) == [24, 12, 12, 12]
    z = np.zeros((4, 4, 4), np.uint8)
    seq, cstep, r2, cnt, st, K = O.invade_literal(z, O.edt(z), 0)
    assert K == 0 and (seq == 0).all() and (cstep == 0).all()
