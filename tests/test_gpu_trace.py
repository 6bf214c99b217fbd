"""Per-batch timing trace of the invasion kernel (ibip_invade_trace): the
records tile the steps in order, both loops appear on a sphere pack, tracing
leaves every output unchanged, and bad arguments are refused."""
import ctypes as C

import numpy as np
import pytest

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


@pytest.mark.parametrize("kind", ["blobs", "spheres"])
def test_trace_tiles_the_steps_and_changes_nothing(ctx, kind):
    rng = np.random.default_rng(17)
    if kind == "blobs":
        img = S.blobs((40, 36, 44), 2.0, 0.6, rng)
    else:
        img = S.sphere_pack((48, 40, 56), 4, 0.45, rng)
    d_img = torch.from_numpy(img).cuda()
    d = ctx.edt(d_img)
    seq0, r20, c0, K0, _ = ctx.invade(d_img, d)
    seq0, r20, c0 = seq0.clone(), r20.clone(), c0.clone()
    buf = torch.full((int(img.astype(bool).sum()) + 1, 8), -7, dtype=torch.int32, device="cuda")
    ctx.invade_trace(buf)
    try:
        seq1, r21, c1, K1, _ = ctx.invade(d_img, d)
    finally:
        ctx.invade_trace(None)
    s = ctx.invade_stats()
    assert K1 == K0 and torch.equal(seq1, seq0) and torch.equal(r21, r20) and torch.equal(c1, c0)
    n = s["trace_batches"]
    assert 0 < n <= buf.shape[0]
    rec = buf.cpu().numpy().astype(np.int64)
    assert np.all(rec[n:] == -7)                       # nothing written past the records
    rec, work = rec[:n, :4], rec[:n, 4:]
    # items taken cover the steps; rows and shells are counted in the main loop only
    assert np.all(work[:, 0] >= rec[:, 1]) and np.all(work[:, 0] <= 64)
    main = rec[:, 3] == 0
    assert np.all(work[main, 1] >= rec[main, 1]) and np.all(work[~main, 1] == rec[~main, 1])
    assert np.all(work[main, 2] >= 1) and np.all(work[~main, 2:] == 0)
    assert rec[0, 0] == 0 and np.all(rec[1:, 0] == np.cumsum(rec[:, 1])[:-1])
    assert rec[:, 1].sum() == K1 and np.all(rec[:, 1] >= 1) and np.all(rec[:, 2] > 0)
    assert set(np.unique(rec[:, 3])) <= {0, 1}
    if kind == "spheres":
        assert (rec[:, 3] == 1).any() and (rec[:, 3] == 0).any()
    # the single-voxel loop only commits steps of radius 1
    r2 = r21.cpu().numpy()
    for f, m, _, loop in rec:
        if loop == 1:
            assert np.all(r2[f:f + m] == 1)
    # the kernel's span gives a plausible SM clock, and covers the batches
    mhz = s["span_cycles"] / s["span_ns"] * 1e3
    assert 300 < mhz < 3000
    assert rec[:, 2].sum() <= s["span_cycles"]
    # a later untraced call writes nothing more
    buf.fill_(-7)
    ctx.invade(d_img, d)
    assert bool((buf == -7).all())


def test_trace_capacity_counts_past_the_end(ctx):
    rng = np.random.default_rng(5)
    img = S.blobs((32, 32, 32), 2.0, 0.6, rng)
    d_img = torch.from_numpy(img).cuda()
    big = torch.full((64, 8), -7, dtype=torch.int32, device="cuda")
    ctx.invade_trace(big[:3])   # capacity 3 inside a larger allocation
    try:
        _, _, _, K, _ = ctx.invade(d_img)
    finally:
        ctx.invade_trace(None)
    s = ctx.invade_stats()
    assert s["trace_batches"] > 3
    b = big.cpu().numpy()
    assert np.all(b[3:] == -7) and np.all(b[:3, 1] >= 1) and b[0, 0] == 0


def test_trace_rejects_bad_arguments(ctx):
    from paper_2101_03240_gb300 import ibip
    L = ibip._lib()
    t = torch.zeros(32, dtype=torch.int32, device="cuda")
    assert L.ibip_invade_trace(None, C.c_void_p(t.data_ptr()), 2) == ibip.ERR_ARG
    assert L.ibip_invade_trace(ctx._h, C.c_void_p(t.data_ptr() + 4), 2) == ibip.ERR_ARG   # misaligned
    assert L.ibip_invade_trace(ctx._h, C.c_void_p(t.data_ptr()), -1) == ibip.ERR_ARG
    assert L.ibip_invade_trace(ctx._h, None, 0) == ibip.OK
