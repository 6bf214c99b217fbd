"""The paper-literal invasion of many images in one launch, one thread-block
cluster per image (ibip_invade_literal_batched): every image's sequence,
insertion steps, radii and insertion counts equal the one-image call and the
oracle bit for bit, for every cluster size and for the tuned choice."""
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


def uneven(seed, n):
    rng = np.random.default_rng(seed)
    imgs = []
    for i in range(n):
        shape = tuple(int(x) for x in rng.integers(5, 40, 3))
        if i % 3 == 0:
            imgs.append(S.blobs(tuple(max(s, 6) for s in shape), rng.uniform(1.2, 3.0), rng.uniform(0.5, 0.75), rng))
        elif i % 3 == 1:
            imgs.append(S.sphere_pack(tuple(max(s, 10) for s in shape), int(rng.integers(2, 5)),
                                      rng.uniform(0.35, 0.5), rng))
        else:
            imgs.append(S.random_image(shape, rng.uniform(0.6, 0.95), rng))
    imgs.append(np.zeros((4, 5, 6), np.uint8))   # no pore at all
    imgs.append(np.ones((7, 3, 9), np.uint8))    # no solid: one tied bucket of +infinity
    return imgs, [int(x) for x in rng.integers(0, 6, len(imgs))]


def same_as_single(ctx, imgs, inlets, res):
    for a, inl, r in zip(imgs, inlets, res):
        dev = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        seq, cst, r2, cnt, K, st = ctx.invade_literal(dev, None, inlet=inl)
        assert r["K"] == K and r["status"] == st
        assert torch.equal(r["seq"], seq) and torch.equal(r["cstep"], cst)
        assert torch.equal(r["step_r2"], r2) and torch.equal(r["step_count"], cnt)


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_every_cluster_size_equals_single_and_oracle(ctx, cluster):
    imgs, inlets = uneven(4100 + cluster, 11)
    ctx.set_literal_cluster(cluster)
    try:
        res, cs = ctx.invade_literal_batched([torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs], inlets)
    finally:
        ctx.set_literal_cluster(0)
    assert cs == cluster
    same_as_single(ctx, imgs, inlets, res)
    for a, inl, r in list(zip(imgs, inlets, res))[:4]:
        seq, cstep, r2, cnt, st, K = O.invade_literal(a, O.edt(a), inl)
        assert r["K"] == K and np.array_equal(r["seq"].cpu().numpy(), seq)
        assert np.array_equal(r["cstep"].cpu().numpy(), cstep) and np.array_equal(r["step_r2"].cpu().numpy(), r2)


def test_tuned_and_automatic_choice(ctx, tmp_path):
    imgs, inlets = uneven(4200, 9)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs]
    res, cs = ctx.invade_literal_batched(dev, inlets)   # automatic, untuned
    assert cs in (1, 2, 4, 8)
    same_as_single(ctx, imgs, inlets, res)
    cache = tmp_path / "tune.txt"
    ctx.set_autotune(True, str(cache))
    try:
        res2, cs2 = ctx.invade_literal_batched(dev, inlets)   # times every size, keeps the fastest
        res3, cs3 = ctx.invade_literal_batched(dev, inlets)   # from the cache
    finally:
        ctx.set_autotune(False)
    assert cs2 in (1, 2, 4, 8, 16) and cs3 == cs2
    assert "lit_b:" in cache.read_text()
    for r, r2 in zip(res, res2):
        assert torch.equal(r["seq"], r2["seq"]) and r["K"] == r2["K"]
    for r, r3 in zip(res, res3):
        assert torch.equal(r["seq"], r3["seq"]) and torch.equal(r["step_r2"], r3["step_r2"])


def test_batch_of_workload_images_and_step_limit(ctx):
    imgs = [S.mixed_image(i, 4000, 32, 96) for i in range(12)]
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs]
    res, cs = ctx.invade_literal_batched(dev, 0)
    same_as_single(ctx, imgs, [0] * len(imgs), res)
    # a step limit stops every image at the same step count as the one-image call
    res, cs = ctx.invade_literal_batched(dev[:3], 0, max_steps=5)
    for a, r in zip(imgs[:3], res):
        seq, cst, r2, cnt, K, st = ctx.invade_literal(torch.from_numpy(a).cuda(), None, inlet=0, max_steps=5)
        assert r["K"] == K and r["status"] == st and torch.equal(r["seq"], seq)
