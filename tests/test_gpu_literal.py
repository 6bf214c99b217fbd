"""Paper-literal invasion (ibip_invade_literal) against the oracle, bit for
bit: sequence image, insertion-point steps, squared radius and insertion
count of every step."""
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


def run_both(ctx, img, inlet, max_steps=None, with_dt2=True):
    d = O.edt(img)
    ref = O.invade_literal(img, d, inlet, max_steps=max_steps)
    dev = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    dt2 = torch.from_numpy(d).cuda() if with_dt2 else None
    got = ctx.invade_literal(dev, dt2, inlet=inlet, max_steps=max_steps)
    return ref, got


def check(ref, got):
    seq, cstep, r2, cnt, st, K = ref
    gseq, gcst, gr2, gcnt, gK, gst = got
    assert gK == K and gst == st
    assert np.array_equal(gseq.cpu().numpy(), seq)
    assert np.array_equal(gcst.cpu().numpy(), cstep)
    assert np.array_equal(gr2.cpu().numpy(), r2)
    assert np.array_equal(gcnt.cpu().numpy(), cnt)


@pytest.mark.parametrize("seed", range(30))
def test_literal_random_small(ctx, seed):
    rng = np.random.default_rng(500 + seed)
    shape = tuple(int(x) for x in rng.integers(1, 24, 3))
    img = S.random_image(shape, rng.uniform(0.3, 0.95), rng)
    check(*run_both(ctx, img, int(rng.integers(0, 6)), with_dt2=bool(seed % 2)))


@pytest.mark.parametrize("seed", range(6))
def test_literal_blobs_and_packs(ctx, seed):
    rng = np.random.default_rng(600 + seed)
    shape = (int(rng.integers(30, 70)), int(rng.integers(30, 70)), int(rng.integers(30, 90)))
    if seed % 2:
        img = S.sphere_pack(shape, int(rng.integers(3, 7)), rng.uniform(0.35, 0.5), rng)
    else:
        img = S.blobs(shape, rng.uniform(2.0, 4.0), rng.uniform(0.5, 0.7), rng)
    check(*run_both(ctx, img, seed % 6))


def test_literal_full_size_workloads(ctx):
    for w in (S.c1_blobs48(), S.c2_spheres200()):
        check(*run_both(ctx, w.image, w.inlet))


def test_literal_edges(ctx):
    check(*run_both(ctx, np.zeros((5, 6, 7), np.uint8), 0))           # all solid
    check(*run_both(ctx, np.ones((6, 5, 33), np.uint8), 1))           # no solid: infinite values
    check(*run_both(ctx, np.ones((1, 1, 1), np.uint8), 4))
    rng = np.random.default_rng(7)
    check(*run_both(ctx, S.random_image((1, 40, 70), 0.8, rng), 2))   # one slice thick
    check(*run_both(ctx, S.tube(60, 6), 0))
    check(*run_both(ctx, S.throat_pore(3, 7, 8), 0))


@pytest.mark.parametrize("limit", [0, 1, 5, 40])
def test_literal_step_limit(ctx, limit):
    rng = np.random.default_rng(9)
    img = S.blobs((30, 30, 30), 2.5, 0.6, rng)
    ref, got = run_both(ctx, img, 0, max_steps=limit)
    check(ref, got)
    assert got[5] == -4   # stopped with candidates left
