"""Batched invasion (ibip_invade_batched): many uneven images in one call
must give, image by image, exactly what the per-image calls give, and what
the oracle gives."""
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


def batch_images():
    rng = np.random.default_rng(77)
    imgs = [S.mixed_image(i, 77000, 8, 40) for i in range(14)]
    imgs.append(np.zeros((5, 7, 9), np.uint8))                        # all solid
    imgs.append(np.ones((6, 5, 33), np.uint8))                        # no solid
    imgs.append(S.random_image((1, 30, 70), 0.8, rng))                # one slice thick
    imgs.append(S.tube(40, 4))
    inlets = [int(x) for x in rng.integers(0, 6, len(imgs))]
    outlets = [int(x) for x in rng.integers(0, 6, len(imgs))]
    return imgs, inlets, outlets


def test_batched_equals_single_and_oracle(ctx):
    imgs, inlets, outlets = batch_images()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs]
    res = ctx.invade_batched(dev, inlets, outlets, trapping=True, curve=True)
    for j, (img, d) in enumerate(zip(imgs, dev)):
        r = res[j]
        assert r["status"] == 0
        dt2 = ctx.edt(d)
        seq, r2, cen, K, st = ctx.invade(d, dt2, inlet=inlets[j])
        tr, so = ctx.trapping(seq, outlets[j])
        Sa, Pc, _ = ctx.pc_curve(so, r2)
        assert r["K"] == K
        assert torch.equal(r["seq"], seq) and torch.equal(r["step_r2"], r2) and torch.equal(r["step_centre"], cen)
        assert torch.equal(r["trapped"], tr) and torch.equal(r["seq_out"], so)
        assert torch.equal(r["S"], Sa) and torch.equal(r["Pc"], Pc)
        if j % 3 == 0:
            dref = O.edt(img)
            sref, r2ref, cref, stref, Kref = O.invade(img, dref, inlet=inlets[j])
            trref, soref = O.trapping(sref, outlets[j])
            assert Kref == r["K"] and np.array_equal(r["seq"].cpu().numpy(), sref)
            assert np.array_equal(r["trapped"].cpu().numpy(), trref)


def test_batched_twice_and_without_trapping(ctx):
    imgs, inlets, _ = batch_images()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs[:6]]
    a = ctx.invade_batched(dev, inlets[:6], trapping=False, curve=False)
    b = ctx.invade_batched(dev[::-1], inlets[:6][::-1], trapping=False, curve=False)[::-1]
    for x, y in zip(a, b):
        assert x["K"] == y["K"] and torch.equal(x["seq"], y["seq"]) and torch.equal(x["step_r2"], y["step_r2"])
