"""Serving (ibip_server_*): jobs admitted by device memory as slots free up,
running concurrently on the slots' streams.  Every result must equal, bit
for bit, what the same image gives alone through the one-image calls, and
the admission rules (arrival order, the arena budget) must hold."""
import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import ibip
    return ibip, ibip.Context(0)


def alone(ctx, d, inlet, outlet):
    dt2 = ctx.edt(d)
    seq, r2, cen, K, st = ctx.invade(d, dt2, inlet=inlet)
    tr, so = ctx.trapping(seq, outlet)
    Sa, Pc, _ = ctx.pc_curve(so, r2)
    torch.cuda.synchronize()
    return dict(K=K, seq=seq, step_r2=r2, step_centre=cen, trapped=tr, seq_out=so, S=Sa, Pc=Pc)


def same(r, a):
    assert r["status"] == 0
    assert r["K"] == a["K"]
    for k in ("seq", "step_r2", "step_centre", "trapped", "seq_out", "S", "Pc"):
        assert torch.equal(r[k], a[k]), k


def mix_images(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    imgs = [S.mixed_image(i, seed, lo, hi) for i in range(n)]
    inl = [int(x) for x in rng.integers(0, 6, n)]
    outl = [int(x) for x in rng.integers(0, 6, n)]
    return imgs, inl, outl


def test_mix_equals_alone_and_admission(lib):
    ibip, ctx = lib
    imgs, inl, outl = mix_images(91000, 16, 12, 56)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs]
    ref = [alone(ctx, d, inl[j], outl[j]) for j, d in enumerate(dev)]
    fp = [ibip.job_footprint(a.shape) for a in imgs]
    budget = int(2.5 * max(fp))   # binds: only a few jobs fit at once
    srv = ibip.Server(ctx, budget, max_slots=6)
    try:
        tickets = [srv.submit(d, inlet=inl[j], outlet=outl[j]) for j, d in enumerate(dev)]
        res = [srv.wait(t, timeout=600) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for j, r in enumerate(res):
        assert r is not None
        same(r, ref[j])
        assert r["mem_used"] <= r["mem_reserved"] == fp[j]
        assert r["t_submit_ns"] <= r["t_start_ns"] <= r["t_end_ns"]
    # arrival order: no job is admitted before an earlier one
    starts = [r["t_start_ns"] for r in res]
    assert starts == sorted(starts)
    assert st["completed"] == len(imgs) and st["running"] == 0 and st["waiting"] == 0
    assert st["arena_used"] == 0 and st["peak_arena_used"] <= budget
    assert st["peak_running"] >= 2


def test_late_arrivals_overlap_a_long_job(lib):
    """Requests that arrive while a long job runs are admitted beside it and
    finish first; the long job's result is unchanged."""
    ibip, ctx = lib
    big = torch.from_numpy(S.blobs((96, 96, 96), 3.0, 0.6, np.random.default_rng(5))).cuda()
    small_np, inl, outl = mix_images(92000, 8, 10, 24)
    small = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in small_np]
    ref_big = alone(ctx, big, 0, 1)
    ref_small = [alone(ctx, d, inl[j], outl[j]) for j, d in enumerate(small)]
    srv = ibip.Server(ctx, 1 << 30, max_slots=4)
    try:
        tb = srv.submit(big, inlet=0, outlet=1)
        ts = [srv.submit(d, inlet=inl[j], outlet=outl[j]) for j, d in enumerate(small)]
        rs = [srv.wait(t, timeout=600) for t in ts]
        rb = srv.wait(tb, timeout=600)
    finally:
        srv.close()
    same(rb, ref_big)
    for j, r in enumerate(rs):
        same(r, ref_small[j])
    assert min(r["t_start_ns"] for r in rs) < rb["t_end_ns"]
    assert len({r["slot"] for r in rs} | {rb["slot"]}) >= 2


def test_edge_images_and_footprint_bound(lib):
    ibip, ctx = lib
    rng = np.random.default_rng(93)
    imgs = [np.zeros((5, 7, 9), np.uint8), np.ones((6, 5, 33), np.uint8), S.random_image((1, 30, 70), 0.8, rng),
            S.tube(40, 4), S.random_image((33, 1, 1), 0.9, rng), S.throat_pore(3, 7, 8)]
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs]
    srv = ibip.Server(ctx, 1 << 28, max_slots=3)
    try:
        ts = [srv.submit(d, inlet=0, outlet=1) for d in dev]
        res = [srv.wait(t, timeout=600) for t in ts]
    finally:
        srv.close()
    for d, r in zip(dev, res):
        same(r, alone(ctx, d, 0, 1))
        assert r["mem_used"] <= r["mem_reserved"]
    # against the oracle on two of them
    for j in (2, 3):
        dref = O.edt(imgs[j])
        sref, _, _, _, Kref = O.invade(imgs[j], dref, inlet=0)
        trref, _ = O.trapping(sref, 1)
        assert res[j]["K"] == Kref
        assert np.array_equal(res[j]["seq"].cpu().numpy(), sref)
        assert np.array_equal(res[j]["trapped"].cpu().numpy(), trref)


def test_job_larger_than_arena_is_refused(lib):
    ibip, ctx = lib
    img = torch.ones((64, 64, 64), dtype=torch.uint8, device="cuda")
    srv = ibip.Server(ctx, ibip.job_footprint((64, 64, 64)) // 2, max_slots=2)
    try:
        with pytest.raises(ibip.IbipError) as e:
            srv.submit(img)
        assert e.value.status == ibip.ERR_OOM
        # the server still serves jobs that fit
        small = torch.from_numpy(S.random_image((16, 16, 16), 0.7, np.random.default_rng(1))).cuda()
        r = srv.wait(srv.submit(small), timeout=600)
        same(r, alone(ctx, small, 0, 1))
    finally:
        srv.close()
