"""Sphere-size image, re-ranked trapping with the surviving steps' radii
feeding the Pc curve, and trapping of the opening's levels (the MIO-vs-IBIP
trapping comparison), bit for bit against the oracle."""
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("seed", range(8))
def test_size_image_and_rerank(ctx, seed):
    rng = np.random.default_rng(1100 + seed)
    shape = tuple(int(x) for x in rng.integers(8, 48, 3))
    img = S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.7), rng) if seed % 2 else \
        S.sphere_pack(shape, int(rng.integers(2, 5)), rng.uniform(0.35, 0.5), rng)
    d = O.edt(img)
    dev = cuda(img)
    seq, r2, cen, K, st = ctx.invade(dev, cuda(d), inlet=seed % 6)
    # every expected value below chains oracle to oracle from the image
    sref, r2ref, _, _, Kref = O.invade(img, d, inlet=seed % 6)
    assert K == Kref and np.array_equal(seq.cpu().numpy(), sref) and np.array_equal(r2.cpu().numpy(), r2ref)
    assert np.array_equal(ctx.size_image(seq, r2).cpu().numpy(), O.size_image(sref, r2ref))
    outlet = (seed + 1) % 6
    tr, so, r2o = ctx.trapping_rerank(seq, r2, outlet)
    rtr, rso, rr2o = O.rerank_radii(sref, r2ref, outlet)
    assert np.array_equal(tr.cpu().numpy(), rtr) and np.array_equal(so.cpu().numpy(), rso)
    assert np.array_equal(r2o.cpu().numpy(), rr2o)
    Sg, Pg, _ = ctx.pc_curve(so, r2o)
    Sr, Pr = O.pc_curve(rso, rr2o)[:2]
    assert np.array_equal(Sg.cpu().numpy(), Sr) and np.array_equal(Pg.cpu().numpy(), Pr)


@pytest.mark.parametrize("seed", range(4))
def test_trapping_of_opening_levels(ctx, seed):
    rng = np.random.default_rng(1200 + seed)
    img = S.sphere_pack((40, 36, 44), 4, 0.4, rng)
    d = O.edt(img)
    T = S.mio_levels(int(d[img > 0].max()), 20)
    dev = cuda(img)
    lev, cnt = ctx.morph_drainage(dev, cuda(d), T, inlet=0)
    lev_ref, cnt_ref = O.morph_drainage(img, d, T, inlet=0)
    assert np.array_equal(lev.cpu().numpy(), lev_ref) and cnt == cnt_ref.tolist()
    tr, so = ctx.trapping(lev, 1)
    rtr, rso = O.trapping(lev_ref, 1)
    assert np.array_equal(tr.cpu().numpy(), rtr) and np.array_equal(so.cpu().numpy(), rso)
