"""ibip_invade_ex: inlet masks (interior inlets) and resuming a run from its
partial sequence, bit for bit against the oracle's uninterrupted runs."""
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


def same(got, ref):
    seq, r2, cen, K, st = got
    rseq, rr2, rcen, rst, rK = ref
    assert K == rK and st == rst
    assert np.array_equal(seq.cpu().numpy(), rseq)
    assert np.array_equal(r2.cpu().numpy(), rr2) and np.array_equal(cen.cpu().numpy(), rcen)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("seed", range(16))
def test_masks(ctx, seed):
    rng = np.random.default_rng(800 + seed)
    shape = tuple(int(x) for x in rng.integers(3, 40, 3))
    img = S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.75), rng) if seed % 2 else \
        S.random_image(shape, rng.uniform(0.4, 0.9), rng)
    d = O.edt(img)
    mask = (rng.random(img.shape) < rng.uniform(0.0005, 0.05)).astype(np.uint8)
    ref = O.invade(img, d, mask=mask)
    same(ctx.invade_ex(cuda(img), cuda(d), inlet_mask=cuda(mask)), ref)


def test_mask_none_is_the_face(ctx):
    rng = np.random.default_rng(5)
    img = S.blobs((30, 28, 33), 2.0, 0.6, rng)
    d = O.edt(img)
    for face in range(6):
        same(ctx.invade_ex(cuda(img), cuda(d), inlet=face), O.invade(img, d, inlet=face))


@pytest.mark.parametrize("seed", range(8))
def test_resume_equals_one_run(ctx, seed):
    rng = np.random.default_rng(900 + seed)
    shape = tuple(int(x) for x in rng.integers(10, 48, 3))
    img = S.sphere_pack(shape, int(rng.integers(2, 5)), rng.uniform(0.35, 0.5), rng) if seed % 2 else \
        S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.75), rng)
    d = O.edt(img)
    mask = None
    if seed % 3 == 2:
        mask = (rng.random(img.shape) < 0.01).astype(np.uint8)
    ref = O.invade(img, d, inlet=seed % 6, mask=mask)
    K = ref[4]
    dm = None if mask is None else cuda(mask)
    cuts = sorted(set(int(c) for c in rng.integers(0, max(K, 1), 3)))
    # the run in chunks ending at each cut, then to the end
    seq, r2, cen, k, st = ctx.invade_ex(cuda(img), cuda(d), inlet=seed % 6, inlet_mask=dm, max_steps=cuts[0])
    assert k == min(cuts[0], K)
    for c in cuts[1:] + [None]:
        extra = None if c is None else c - k
        seq, r2, cen, k, st = ctx.invade_ex(cuda(img), cuda(d), inlet=seed % 6, inlet_mask=dm,
                                            resume_from=(seq, r2, cen), max_steps=extra)
    same((seq, r2, cen, k, st), ref)


def test_resume_a_finished_run_and_full_size(ctx):
    w = S.c2_spheres200()
    d = O.edt(w.image)
    ref = O.invade(w.image, d, inlet=0)
    img, dd = cuda(w.image), cuda(d)
    half = ref[4] // 2
    seq, r2, cen, k, st = ctx.invade_ex(img, dd, max_steps=half)
    assert k == half and st == -4
    got = ctx.invade_ex(img, dd, resume_from=(seq, r2, cen))
    same(got, ref)
    again = ctx.invade_ex(img, dd, resume_from=got[:3])
    same(again, ref)
