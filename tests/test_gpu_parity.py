"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element on the same seeded inputs.  Integer outputs (dt2, seq,
step arrays, trapped mask, levels, counts) must be bit-exact; saturation and
Pc must be bit-exact too (same double formula, one rounding to float), which
is stricter than the 1e-6 relative bound the method is held to."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import ibip
    return ibip.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def rand_case(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in rng.integers(1, 48, 3))
    if seed % 4 == 0:
        shape = tuple(max(s, 6) for s in shape)
        img = S.blobs(shape, rng.uniform(1.0, 3.0), rng.uniform(0.4, 0.8), rng)
    elif seed % 4 == 1:
        img = S.random_image(shape, rng.uniform(0.5, 0.97), rng)
    elif seed % 4 == 2:
        shape = tuple(max(s, 12) for s in shape)
        img = S.sphere_pack(shape, int(rng.integers(2, 6)), rng.uniform(0.35, 0.6), rng)
    else:
        img = S.random_image(shape, 0.99, rng)
    return img, int(rng.integers(0, 6)), int(rng.integers(0, 6))


# ------------------------------------------------------------------ EDT ----

@pytest.mark.parametrize("seed", range(24))
def test_edt_random(ctx, seed):
    img, _, _ = rand_case(seed)
    assert np.array_equal(host(ctx.edt(dev(img))), O.edt(img))


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 70), (70, 1, 1), (1, 70, 1), (33, 2, 65), (5, 129, 31),
                                   (1, 1700, 3), (1700, 2, 3)])
def test_edt_thin_and_degenerate(ctx, shape):
    rng = np.random.default_rng(sum(shape))
    for img in (S.random_image(shape, 0.8, rng), np.ones(shape, np.uint8), np.zeros(shape, np.uint8)):
        assert np.array_equal(host(ctx.edt(dev(img))), O.edt(img))


def test_edt_single_solid_far_field(ctx):
    img = np.ones((40, 33, 70), np.uint8)
    img[3, 30, 1] = 0
    assert np.array_equal(host(ctx.edt(dev(img))), O.edt_brute(img))


def test_edt_configs(ctx):
    for w in (S.c1_blobs48(), S.c2_spheres200()):
        assert np.array_equal(host(ctx.edt(dev(w.image))), O.edt(w.image)), w.name


# ------------------------------------------------------------- invasion ----

def check_invade(ctx, img, inlet, **kw):
    d = O.edt(img)
    ref = O.invade(img, d, inlet=inlet, **kw)
    seq, r2, cen, K, st = ctx.invade(dev(img), dev(d), inlet=inlet, **kw)
    assert K == ref[4] and st == ref[3]
    assert np.array_equal(host(seq), ref[0])
    assert np.array_equal(host(r2), ref[1])
    assert np.array_equal(host(cen), ref[2])
    return ref


@pytest.mark.parametrize("case", ["row_ties", "slab_front"])
def test_invade_hand_examples(ctx, case):
    g = GOLD[case]
    img = np.array(g["image"], np.uint8)
    seq, r2, cen, K, st = ctx.invade(dev(img), None, inlet=g["inlet"])
    assert np.array_equal(host(seq), np.array(g["seq"], np.int32))
    assert host(r2).tolist() == g["step_r2"] and host(cen).tolist() == g["step_centre"]


@pytest.mark.parametrize("seed", range(40))
def test_invade_random(ctx, seed):
    img, inlet, _ = rand_case(1000 + seed)
    check_invade(ctx, img, inlet)


def test_invade_degenerate(ctx):
    check_invade(ctx, np.zeros((5, 6, 7), np.uint8), 0)
    check_invade(ctx, np.ones((9, 8, 37), np.uint8), 0)         # no solid: one step
    img = np.ones((9, 9, 9), np.uint8)
    img[:, :, 0] = 0
    check_invade(ctx, img, 4)                                    # inlet face all solid
    check_invade(ctx, np.ones((1, 1, 1), np.uint8), 3)
    check_invade(ctx, S.tube(60, 7), 0)
    check_invade(ctx, S.throat_pore(3, 9, 6), 0)


def test_invade_step_limit_and_capacity(ctx):
    img = S.blobs((30, 31, 29), 2.0, 0.6, np.random.default_rng(3))
    for ms in (0, 1, 7, 100):
        check_invade(ctx, img, 0, max_steps=ms)
    d = O.edt(img)
    ref = O.invade(img, d)
    seq, r2, cen, K, st = ctx.invade(dev(img), dev(d), capacity=5, check=False)
    assert st == -1 and K == ref[4] and np.array_equal(host(seq), ref[0])
    assert np.array_equal(host(r2), ref[1][:5])


def test_invade_c1(ctx):
    w = S.c1_blobs48()
    check_invade(ctx, w.image, w.inlet)


def test_invade_c2(ctx):
    w = S.c2_spheres200()
    check_invade(ctx, w.image, w.inlet)


def test_invade_dt2_computed_inside(ctx):
    img, inlet, _ = rand_case(77)
    d = O.edt(img)
    ref = O.invade(img, d, inlet=inlet)
    seq, r2, cen, K, st = ctx.invade(dev(img), None, inlet=inlet)
    assert np.array_equal(host(seq), ref[0]) and np.array_equal(host(r2), ref[1])


# ------------------------------------------------------------- trapping ----

@pytest.mark.parametrize("case", ["trap_same_step", "trap_row", "trap_pocket_rerank"])
def test_trap_hand_examples(ctx, case):
    g = GOLD[case]
    seq = np.array(g["seq"], np.int32)
    tr, so = ctx.trapping(dev(seq), g["outlet"], rerank="seq_out_rerank" in g)
    assert np.array_equal(host(tr), np.array(g["trapped"], np.uint8))
    if "seq_out_rerank" in g:
        assert np.array_equal(host(so), np.array(g["seq_out_rerank"], np.int32))


@pytest.mark.parametrize("seed", range(20))
def test_trap_random(ctx, seed):
    img, inlet, outlet = rand_case(2000 + seed)
    seq = O.invade(img, O.edt(img), inlet=inlet)[0]
    for rr in (False, True):
        tr_ref, so_ref = O.trapping(seq, outlet, rerank=rr)
        tr, so = ctx.trapping(dev(seq), outlet, rerank=rr)
        assert np.array_equal(host(tr), tr_ref) and np.array_equal(host(so), so_ref)


def test_trap_c2(ctx):
    w = S.c2_spheres200()
    seq = O.invade(w.image, O.edt(w.image))[0]
    tr_ref, so_ref = O.trapping(seq, w.outlet)
    tr, so = ctx.trapping(dev(seq), w.outlet)
    assert np.array_equal(host(tr), tr_ref) and np.array_equal(host(so), so_ref)


# ------------------------------------------------------------------- Pc ----

def test_pc_hand_example(ctx):
    g = GOLD["pc_small"]
    seq = np.array(g["seq"], np.int32)
    Sa, Pc, img = ctx.pc_curve(dev(seq), dev(np.array(g["step_r2"], np.int32)), g["voxel_m"], g["sigma"],
                               g["theta_deg"], sat_image=True)
    assert host(Sa).tolist() == g["S"]
    np.testing.assert_allclose(host(Pc), g["Pc"], rtol=1e-6)
    assert host(img).ravel().tolist() == [0.5, 0.5, 0.75, 1.0, float("inf")]


@pytest.mark.parametrize("seed", range(8))
def test_pc_random(ctx, seed):
    img, inlet, outlet = rand_case(3000 + seed)
    seq, r2, _, _, K = O.invade(img, O.edt(img), inlet=inlet)
    th = [180.0, 150.0, 95.0, 120.0][seed % 4]
    Sr, Pr, Ir = O.pc_curve(seq, r2, 4e-6, 0.05, th, sat_image=True)
    Sg, Pg, Ig = ctx.pc_curve(dev(seq), dev(r2), 4e-6, 0.05, th, sat_image=True)
    assert np.array_equal(host(Sg), Sr) and np.array_equal(host(Ig), Ir)
    np.testing.assert_allclose(host(Pg), Pr, rtol=1e-6)
    assert np.array_equal(host(Pg), Pr)


# --------------------------------------------------------- opening (MIO) ----

def test_mio_hand_example(ctx):
    g = GOLD["mio_slab"]
    img = np.array(g["image"], np.uint8)
    d = O.edt(img)
    lev, cnt = ctx.morph_drainage(dev(img), dev(d), g["levels"], inlet=g["inlet"])
    assert np.array_equal(host(lev), np.array(g["level"], np.int32)) and cnt == g["counts"]


@pytest.mark.parametrize("seed", range(12))
def test_mio_random(ctx, seed):
    img, inlet, _ = rand_case(4000 + seed)
    d = O.edt(img)
    if not (img == 1).any() or (d == np.iinfo(np.int32).max).any():
        return
    T = S.mio_levels(int(d[img == 1].max()), 12)
    lev_ref, cnt_ref = O.morph_drainage(img, d, T, inlet=inlet)
    lev, cnt = ctx.morph_drainage(dev(img), dev(d), T, inlet=inlet)
    assert np.array_equal(host(lev), lev_ref) and cnt == cnt_ref.tolist()


def test_mio_c1(ctx):
    w = S.c1_blobs48()
    d = O.edt(w.image)
    T = S.mio_levels(int(d.max()), 40)
    lev_ref, cnt_ref = O.morph_drainage(w.image, d, T, inlet=0)
    lev, cnt = ctx.morph_drainage(dev(w.image), dev(d), T, inlet=0)
    assert np.array_equal(host(lev), lev_ref) and cnt == cnt_ref.tolist()
