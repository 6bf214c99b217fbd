"""Pins for the CPU oracle: hand-worked cases, closed forms, a library
routine, brute force and invariants.  None of these compare the oracle with
itself: each fixes what the paper's definitions force, so that a dropped
term, a wrong sign, a swapped axis or a wrong tie/strictness rule in the
oracle fails at least one test.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))
INT32_MAX = np.iinfo(np.int32).max


def arr(x, dt):
    return np.array(x, dtype=dt)


# ---------------------------------------------------------------- EDT ----

def scipy_dt2(img):
    from scipy.ndimage import distance_transform_edt
    return np.rint(distance_transform_edt(img) ** 2).astype(np.int64)


@pytest.mark.parametrize("seed", range(12))
def test_edt_brute_matches_scipy_and_sep(seed):
    """Section 2.1 'distance transform': EDT-brute equals SciPy's exact EDT
    squared (outside the image is not solid in both), and EDT-sep equals
    EDT-brute, on anisotropic shapes so a swapped axis shows."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in rng.integers(3, 12, 3))
    img = S.random_image(shape, rng.uniform(0.3, 0.95), rng)
    img[tuple(rng.integers(0, s) for s in shape)] = 0
    b = O.edt_brute(img)
    assert np.array_equal(b, scipy_dt2(img))
    assert np.array_equal(O.edt(img), b)


def test_edt_special_cases():
    # single solid voxel: dt2 = |v - s|^2 everywhere
    img = np.ones((7, 5, 9), np.uint8)
    s = (2, 4, 1)
    img[s] = 0
    x, y, z = np.indices(img.shape)
    want = (x - s[0]) ** 2 + (y - s[1]) ** 2 + (z - s[2]) ** 2
    assert np.array_equal(O.edt(img), want)
    assert np.array_equal(O.edt_brute(img), want)
    # half-space solid x >= 6: dt2 = (6 - x)^2 on pore
    img = np.ones((9, 4, 5), np.uint8)
    img[6:] = 0
    xi = np.indices(img.shape)[0]
    want = np.where(xi < 6, (6 - xi) ** 2, 0)
    assert np.array_equal(O.edt(img), want)
    # all solid -> 0; no solid -> INT32_MAX
    assert not O.edt(np.zeros((3, 4, 5), np.uint8)).any()
    assert (O.edt(np.ones((3, 4, 5), np.uint8)) == INT32_MAX).all()
    assert (O.edt_brute(np.ones((2, 2, 2), np.uint8)) == INT32_MAX).all()


def test_edt_hand_examples():
    for k in ("row_ties", "slab_front"):
        g = GOLD[k]
        assert np.array_equal(O.edt(arr(g["image"], np.uint8)), arr(g["dt2"], np.int32))


# ----------------------------------------------------------- invasion ----

@pytest.mark.parametrize("case", ["row_ties", "slab_front"])
@pytest.mark.parametrize("method", ["scan", "heap"])
def test_invade_hand_examples(case, method):
    """Section 2.1: hand-worked sequences (tie rule, candidate rule)."""
    g = GOLD[case]
    img = arr(g["image"], np.uint8)
    seq, r2, cen, st, K = O.invade(img, O.edt(img), inlet=g["inlet"], method=method)
    assert st == O.OK and K == len(g["step_r2"])
    assert np.array_equal(seq, arr(g["seq"], np.int32))
    assert r2.tolist() == g["step_r2"] and cen.tolist() == g["step_centre"]


@pytest.mark.parametrize("R,nx", [(3, 20), (5, 31), (8, 50), (1, 6), (2, 9)])
def test_invade_tube_closed_form(R, nx):
    """Straight tube of integer radius R along x, inlet X0: the axis has
    dt2 = R^2 exactly (the solid at (R,0) in the cross-section), so the
    first ceil(nx/R) steps put centres at (jR, cy, cz) with r2 = R^2; voxel p
    inside the tube gets the first j with (x - jR)^2 + rho^2 < R^2; the first
    outlet-face voxel falls at step ceil(nx/R).  A '<=' stamp or a
    non-strict tie would move the centres."""
    img = S.tube(nx, R)
    n = img.shape[1]
    c = n // 2
    d = O.edt(img)
    assert d[:, c, c].tolist() == [R * R] * nx
    seq, r2, cen, st, K = O.invade(img, d, inlet=0)
    J = math.ceil(nx / R)
    assert r2[:J].tolist() == [R * R] * J
    assert cen[:J].tolist() == [((j * R) * n + c) * n + c for j in range(J)]
    x, y, z = np.indices(img.shape)
    rho2 = (y - c) ** 2 + (z - c) ** 2
    want = np.full(img.shape, -2)
    for j in range(J - 1, -1, -1):
        inside = ((x - j * R) ** 2 + rho2 < R * R) & (img == 1)
        want[inside] = j + 1
    m = want > 0
    assert np.array_equal(seq[m], want[m])
    assert seq[nx - 1][img[nx - 1] == 1].min() == J
    # breakthrough pressure: 2 sigma / (R voxel); R=8, 5 um, 0.072 N/m -> 3600 Pa
    Sat, Pc, _ = O.pc_curve(seq, r2, 5e-6, 0.072, 180.0)
    assert Pc[J - 1] == np.float32(2 * 0.072 / (R * 5e-6))
    if R == 8:
        assert Pc[J - 1] == np.float32(3600.0)


@pytest.mark.parametrize("rt,rp,lt", [(2, 6, 5), (3, 8, 7), (2, 9, 6)])
def test_invade_throat_pore_jump(rt, rp, lt):
    """Pore behind a throat (Section 2.2.2: the meniscus breaches a
    constriction, then the pressure drops while the cavity fills).  Before
    the first centre inside the pore body the smallest step radius is the
    throat's (max Pc = 2 sigma / r_t); the first centre in the body has a
    larger r2 (the jump)."""
    img = S.throat_pore(rt, rp, lt)
    d = O.edt(img)
    seq, r2, cen, st, K = O.invade(img, d, inlet=0)
    nx, n = img.shape[0], img.shape[1]
    c = n // 2
    cx = lt + rp
    cc = np.array(np.unravel_index(cen, img.shape)).T
    in_body = ((cc[:, 0] - cx) ** 2 + (cc[:, 1] - c) ** 2 + (cc[:, 2] - c) ** 2 < (rp - rt) ** 2)
    first = int(np.flatnonzero(in_body)[0])
    assert r2[:first].min() == rt * rt
    assert r2[first] > rt * rt
    # running max of Pc equals the throat's while the body fills
    Sat, Pc, _ = O.pc_curve(seq, r2)
    runmax = np.maximum.accumulate(Pc)
    assert runmax[first] == np.float32(2 * 0.072 / (rt * 5e-6))


def front_max_scan(seq, d, img, inlet):
    """Largest dt2 over the current candidate set (brute force)."""
    cand = (seq == -1)
    inv = np.pad(seq >= 1, 1)
    nb = inv[:-2, 1:-1, 1:-1] | inv[2:, 1:-1, 1:-1] | inv[1:-1, :-2, 1:-1] | \
        inv[1:-1, 2:, 1:-1] | inv[1:-1, 1:-1, :-2] | inv[1:-1, 1:-1, 2:]
    face = np.zeros_like(cand)
    sl = [slice(None)] * 3
    sl[inlet // 2] = 0 if inlet % 2 == 0 else -1
    face[tuple(sl)] = True
    cand &= (nb | face)
    return d[cand].max() if cand.any() else None


@pytest.mark.parametrize("seed", range(40))
def test_invade_scan_equals_heap_and_invariants(seed):
    """Invade-scan (the definition) equals invade-heap bit for bit; the
    invariants hold: every voxel of step k lies in ball(c_k, r2_k); stamped
    voxels are pore; r2_k is the largest dt2 over the candidates before
    step k; every invaded voxel reaches the inlet through voxels invaded no
    later; the invaded set is the inlet-connected pore component."""
    from scipy.ndimage import label
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(s) for s in rng.integers(4, 11, 3))
    if seed % 3 == 0:
        img = S.blobs(shape, rng.uniform(0.8, 2.0), rng.uniform(0.4, 0.8), rng)
    else:
        img = S.random_image(shape, rng.uniform(0.45, 0.95), rng)
    inlet = int(rng.integers(0, 6))
    d = O.edt(img)
    a = O.invade(img, d, inlet=inlet, method="scan")
    b = O.invade(img, d, inlet=inlet, method="heap")
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
    seq, r2, cen, st, K = a
    assert st == O.OK and K == len(r2)
    assert ((seq >= 1) <= (img == 1)).all()
    pos = np.indices(img.shape).reshape(3, -1).T
    flat = seq.ravel()
    for k in range(1, K + 1):
        c = np.array(np.unravel_index(cen[k - 1], img.shape))
        m = flat == k
        assert m[cen[k - 1]]
        dd = ((pos[m] - c) ** 2).sum(1)
        assert (dd < r2[k - 1]).all()
        assert r2[k - 1] == d.ravel()[cen[k - 1]]
    # r2_k is the front maximum: replay the thresholded sequence
    for k in range(1, K + 1):
        before = np.where((seq >= 1) & (seq < k), seq, np.where(img == 1, -1, 0))
        assert front_max_scan(before, d, img, inlet) == r2[k - 1]
    assert O.count_unconnected(seq, inlet) == 0
    lab, _ = label(img, structure=[[[0, 0, 0], [0, 1, 0], [0, 0, 0]],
                                   [[0, 1, 0], [1, 1, 1], [0, 1, 0]],
                                   [[0, 0, 0], [0, 1, 0], [0, 0, 0]]])
    sl = [slice(None)] * 3
    sl[inlet // 2] = 0 if inlet % 2 == 0 else -1
    ids = np.unique(lab[tuple(sl)])
    reach = np.isin(lab, ids[ids > 0])
    assert np.array_equal(seq >= 1, reach)


def test_invade_degenerate():
    # all solid: nothing to do
    img = np.zeros((3, 4, 5), np.uint8)
    seq, r2, cen, st, K = O.invade(img, O.edt(img))
    assert K == 0 and not seq.any()
    # no solid: one step invades everything (dt2 = INT32_MAX, ball clamped)
    img = np.ones((4, 3, 5), np.uint8)
    seq, r2, cen, st, K = O.invade(img, O.edt(img), inlet=0)
    assert K == 1 and (seq == 1).all() and r2[0] == INT32_MAX and cen[0] == 0
    # inlet face all solid: nothing enters
    img = np.ones((5, 5, 5), np.uint8)
    img[0] = 0
    seq, r2, cen, st, K = O.invade(img, O.edt(img), inlet=0)
    assert K == 0 and (seq[1:] == -1).all()
    # nx = 1, single voxel
    img = np.ones((1, 1, 1), np.uint8)
    seq, r2, cen, st, K = O.invade(img, O.edt(img), inlet=3)
    assert K == 1 and seq[0, 0, 0] == 1


def test_invade_step_limit_and_capacity():
    rng = np.random.default_rng(7)
    img = S.random_image((8, 8, 8), 0.7, rng)
    d = O.edt(img)
    full = O.invade(img, d)
    K = full[4]
    assert K > 5
    part = O.invade(img, d, max_steps=5)
    assert part[3] == O.STEP_LIMIT and part[4] == 5
    assert np.array_equal(part[1], full[1][:5])
    assert np.array_equal(np.where(full[0] > 5, -1, full[0]), part[0])
    small = O.invade(img, d, capacity=3)
    assert small[4] == K and len(small[1]) == 3 and np.array_equal(small[0], full[0])
    exact = O.invade(img, d, max_steps=K)
    assert exact[3] == O.OK and exact[4] == K


# ----------------------------------------------------------- trapping ----

@pytest.mark.parametrize("case", ["trap_same_step", "trap_row", "trap_pocket_rerank"])
@pytest.mark.parametrize("method", ["bfs", "uf"])
def test_trap_hand_examples(case, method):
    g = GOLD[case]
    seq = arr(g["seq"], np.int32)
    tr, out = O.trapping(seq, g["outlet"], rerank="seq_out_rerank" in g, method=method)
    assert np.array_equal(tr, arr(g["trapped"], np.uint8))
    if "seq_out_rerank" in g:
        assert np.array_equal(out, arr(g["seq_out_rerank"], np.int32))
    else:
        assert np.array_equal(out, np.where(tr == 1, -1, seq))


@pytest.mark.parametrize("seed", range(25))
def test_trap_bfs_equals_uf(seed):
    """Section 2.2.3: the per-threshold flood (definition) and the one-pass
    reverse union-find agree; trapped voxels are invaded; outlet-face voxels
    are never trapped; a voxel on a path of non-decreasing sequence to the
    outlet is not trapped."""
    rng = np.random.default_rng(500 + seed)
    shape = tuple(int(s) for s in rng.integers(4, 10, 3))
    img = S.random_image(shape, rng.uniform(0.5, 0.95), rng)
    inlet = int(rng.integers(0, 6))
    outlet = int(rng.integers(0, 6))
    seq = O.invade(img, O.edt(img), inlet=inlet)[0]
    a = O.trapping(seq, outlet, rerank=bool(seed % 2), method="bfs")
    b = O.trapping(seq, outlet, rerank=bool(seed % 2), method="uf")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    tr = a[0].astype(bool)
    assert (seq[tr] >= 1).all()
    sl = [slice(None)] * 3
    sl[outlet // 2] = 0 if outlet % 2 == 0 else -1
    assert not tr[tuple(sl)].any()
    if seed % 2:
        kept = np.unique(a[1][a[1] >= 1])
        assert kept.tolist() == list(range(1, len(kept) + 1))


def test_trap_no_solid_and_random_walks():
    img = np.ones((6, 5, 4), np.uint8)
    seq = O.invade(img, O.edt(img))[0]
    assert not O.trapping(seq, 1)[0].any()
    # monotone sequence towards the outlet: nothing trapped
    seq = np.arange(1, 11, dtype=np.int32).reshape(10, 1, 1)
    assert not O.trapping(seq, 1)[0].any()
    # decreasing towards the outlet: everything but the outlet voxel trapped
    seq = np.arange(10, 0, -1, dtype=np.int32).reshape(10, 1, 1).copy()
    tr = O.trapping(seq, 1)[0].ravel()
    assert tr.tolist() == [1] * 9 + [0]


# ---------------------------------------------------------------- MIO ----

@pytest.mark.parametrize("method", ["plain", "edt"])
def test_mio_hand_example(method):
    g = GOLD["mio_slab"]
    img = arr(g["image"], np.uint8)
    lev, cnt = O.morph_drainage(img, O.edt(img), g["levels"], inlet=g["inlet"], method=method)
    assert np.array_equal(lev, arr(g["level"], np.int32))
    assert cnt.tolist() == g["counts"]


@pytest.mark.parametrize("R", [2, 4, 6])
def test_mio_tube_closed_form(R):
    """A tube of radius R admits the sphere d^2 < R^2 along its whole axis,
    which then sweeps the whole tube; a larger sphere does not fit."""
    img = S.tube(15, R)
    d = O.edt(img)
    T = [R * R + 3, R * R + 1, R * R]
    for method in ("plain", "edt"):
        lev, cnt = O.morph_drainage(img, d, T, inlet=0, method=method)
        assert cnt.tolist() == [0, 0, int(img.sum())]
        assert (lev[img == 1] == 3).all()


@pytest.mark.parametrize("rt,rp,lt", [(2, 6, 4), (3, 7, 5)])
def test_mio_trims_before_dilation(rt, rp, lt):
    """Section 2.4.1: a pore body behind a throat is not reached at any
    sphere larger than the throat: after the erosion the body is cut off
    from the inlet and trimmed."""
    img = S.throat_pore(rt, rp, lt)
    d = O.edt(img)
    T = [(rp - 1) ** 2, rt * rt + 1, rt * rt]
    for method in ("plain", "edt"):
        lev, cnt = O.morph_drainage(img, d, T, inlet=0, method=method)
        assert cnt[0] == 0 and cnt[1] == 0 and cnt[2] > 0


@pytest.mark.parametrize("seed", range(8))
def test_mio_plain_equals_edt(seed):
    rng = np.random.default_rng(900 + seed)
    shape = tuple(int(s) for s in rng.integers(6, 14, 3))
    img = S.blobs(shape, rng.uniform(1.0, 2.0), rng.uniform(0.5, 0.8), rng)
    d = O.edt(img)
    T = S.mio_levels(int(d[img == 1].max()), 10)
    a = O.morph_drainage(img, d, T, inlet=0, method="plain")
    b = O.morph_drainage(img, d, T, inlet=0, method="edt")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ----------------------------------------------------------------- Pc ----

def test_pc_hand_example():
    g = GOLD["pc_small"]
    Sat, Pc, img = O.pc_curve(arr(g["seq"], np.int32), g["step_r2"], g["voxel_m"], g["sigma"],
                              g["theta_deg"], sat_image=True)
    assert Sat.tolist() == g["S"]
    np.testing.assert_allclose(Pc, g["Pc"], rtol=1e-6)
    assert img.ravel().tolist() == [0.5, 0.5, 0.75, 1.0, float("inf")]


@pytest.mark.parametrize("seed", range(5))
def test_pc_curve_closed_form(seed):
    """S_k is the cumulative count over all pore voxels; Pc_k is
    -2 sigma cos(theta) / (sqrt(r2_k) * voxel), one rounding to float32
    (independent Python double evaluation); S is non-decreasing."""
    rng = np.random.default_rng(seed)
    img = S.random_image((9, 8, 7), 0.7, rng)
    seq, r2, cen, st, K = O.invade(img, O.edt(img))
    vox, sig, th = 5e-6, 0.072, [180.0, 140.0, 120.0][seed % 3]
    Sat, Pc, _ = O.pc_curve(seq, r2, vox, sig, th)
    npore = int((seq != 0).sum())
    cnt = np.bincount(seq[seq >= 1], minlength=K + 1)[1:]
    want_S = [np.float32(c / npore) for c in np.cumsum(cnt)]
    ct = math.cos(th * math.pi / 180.0)
    want_P = [np.float32((-2.0 * sig * ct) / (math.sqrt(float(r)) * vox)) for r in r2]
    assert Sat.tolist() == want_S and Pc.tolist() == want_P
    assert (np.diff(Sat) >= 0).all()
