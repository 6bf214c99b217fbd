"""Equal-saturation comparison (ibip_equal_saturation) against the oracle's
definition, on invasions of both rules and their opening levels."""
import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import ibip
    return ibip.Context(0)


def compare(ctx, img, inlet, n_levels, rule):
    dev = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    d = ctx.edt(dev)
    if rule == "paper":
        seq, _, r2, _, K, st = ctx.invade_literal(dev, d, inlet=inlet)
    else:
        seq, r2, cen, K, st = ctx.invade(dev, d, inlet=inlet)
    dmax = int(d[dev > 0].max().item()) if bool((dev > 0).any()) else 1
    T = S.mio_levels(min(dmax, 1 << 30), n_levels)
    lev, cnt = ctx.morph_drainage(dev, d, T, inlet=inlet)
    k, diff, n = ctx.equal_saturation(seq, lev, K, len(T))
    rk, rdiff, rn = O.equal_saturation(seq.cpu().numpy(), lev.cpu().numpy(), len(T))
    assert list(rk) == k and list(rdiff) == diff and list(rn) == n
    assert n == cnt
    return k, diff, n


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("rule", ["frontier", "paper"])
def test_equal_saturation_random(ctx, seed, rule):
    rng = np.random.default_rng(700 + seed)
    shape = tuple(int(x) for x in rng.integers(6, 40, 3))
    img = S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.75), rng) if seed % 2 else \
        S.sphere_pack(shape, int(rng.integers(2, 5)), rng.uniform(0.35, 0.5), rng)
    compare(ctx, img, seed % 6, int(rng.integers(1, 60)), rule)


def test_equal_saturation_blobs48_against_oracle_inputs(ctx):
    w = S.c1_blobs48()
    d = O.edt(w.image)
    seq = O.invade(w.image, d, inlet=0)[0]
    T = S.mio_levels(int(d[w.image > 0].max()), 40)
    level = O.morph_drainage(w.image, d, T, inlet=0)[0]
    k, diff, n = ctx.equal_saturation(torch.from_numpy(seq).cuda(), torch.from_numpy(level).cuda(),
                                      int(seq.max()), len(T))
    rk, rdiff, rn = O.equal_saturation(seq, level, len(T))
    assert list(rk) == k and list(rdiff) == diff and list(rn) == n


def test_equal_saturation_edges(ctx):
    z = np.zeros((4, 5, 6), np.uint8)
    dev = torch.from_numpy(z).cuda()
    seq = torch.zeros(z.shape, dtype=torch.int32, device="cuda")
    k, diff, n = ctx.equal_saturation(seq, seq.clone(), 0, 3)
    assert k == [0, 0, 0] and diff == [0, 0, 0] and n == [0, 0, 0]
    compare(ctx, np.ones((5, 4, 7), np.uint8), 0, 5, "frontier")


@pytest.mark.parametrize("seed", range(8))
def test_matched_opening_random(ctx, seed):
    """The opening with the paper-literal closed ball (ibip_morph_drainage_ex,
    erosion R^2, dilation |d|^2 <= R^2 for integer R) against the oracle."""
    rng = np.random.default_rng(900 + seed)
    shape = tuple(int(x) for x in rng.integers(6, 44, 3))
    img = S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.75), rng) if seed % 2 else \
        S.sphere_pack(shape, int(rng.integers(2, 6)), rng.uniform(0.35, 0.5), rng)
    d = O.edt(img)
    Te, Td = S.integer_radius_levels(int(d[img > 0].max()) if img.any() else 1)
    dev = torch.from_numpy(img).cuda()
    lev, cnt = ctx.morph_drainage(dev, torch.from_numpy(d).cuda(), Te, inlet=seed % 6, dilate_levels=Td)
    rlev, rcnt = O.morph_drainage(img, d, Te, inlet=seed % 6, dilate_levels=Td)
    assert np.array_equal(lev.cpu().numpy(), rlev) and cnt == rcnt.tolist()


def test_matched_opening_spheres200(ctx):
    w = S.c2_spheres200()
    d = O.edt(w.image)
    Te, Td = S.integer_radius_levels(int(d[w.image > 0].max()))
    lev, cnt = ctx.morph_drainage(torch.from_numpy(w.image).cuda(), torch.from_numpy(d).cuda(), Te, inlet=0,
                                  dilate_levels=Td)
    rlev, rcnt = O.morph_drainage(w.image, d, Te, inlet=0, dilate_levels=Td)
    assert np.array_equal(lev.cpu().numpy(), rlev) and cnt == rcnt.tolist()


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("rule", ["frontier", "paper"])
def test_pc_envelope_random(ctx, seed, rule):
    """The drainage envelope at opening levels (ibip_pc_envelope) against
    the oracle, on both rules' invasions (the paper rule with its integer
    radius levels)."""
    rng = np.random.default_rng(1300 + seed)
    shape = tuple(int(x) for x in rng.integers(6, 40, 3))
    img = S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.75), rng) if seed % 2 else \
        S.sphere_pack(shape, int(rng.integers(2, 5)), rng.uniform(0.35, 0.5), rng)
    dev = torch.from_numpy(img).cuda()
    d = ctx.edt(dev)
    if rule == "paper":
        seq, _, r2, _, K, st = ctx.invade_literal(dev, d, inlet=seed % 6)
    else:
        seq, r2, cen, K, st = ctx.invade(dev, d, inlet=seed % 6)
    dmax = int(d[dev > 0].max().item()) if bool((dev > 0).any()) else 1
    T = S.integer_radius_levels(dmax)[0] if rule == "paper" else S.mio_levels(dmax, int(rng.integers(1, 60)))
    ks, ns = ctx.pc_envelope(seq, r2, T)
    rk, rn = O.pc_envelope(seq.cpu().numpy(), r2.cpu().numpy(), T)
    assert ks == list(rk) and ns == list(rn)


def test_pc_envelope_blobs48_and_empty(ctx):
    w = S.c1_blobs48()
    d = O.edt(w.image)
    seq, r2, cen, st, K = O.invade(w.image, d, inlet=0)
    T = S.mio_levels(int(d[w.image > 0].max()), 40)
    ks, ns = ctx.pc_envelope(torch.from_numpy(seq).cuda(), torch.from_numpy(r2).cuda(), T)
    rk, rn = O.pc_envelope(seq, r2, T)
    assert ks == list(rk) and ns == list(rn)
    z = torch.zeros((3, 4, 5), dtype=torch.int32, device="cuda")
    assert ctx.pc_envelope(z, torch.zeros(0, dtype=torch.int32, device="cuda"), [4, 1]) == ([0, 0], [0, 0])
