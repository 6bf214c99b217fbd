"""Serving replicas (ibip_router_*): requests routed over several servers,
here two replicas on the one GPU of this machine (a device may be listed
more than once).  Every result must equal what the image gives alone
through the one-image calls, both replicas must take requests, and the
routing must follow the least-outstanding-work rule."""
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


def test_two_replicas_on_one_gpu(lib):
    ibip, ctx = lib
    # the first request is large enough (a 100^3 pack: tens of ms) that the
    # second is routed while it still runs
    imgs = [S.sphere_pack((100, 100, 100), 4, 0.4, np.random.default_rng(93))] + \
        [S.mixed_image(i, 93000, 16, 64) for i in range(13)]
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in imgs]
    ref = [alone(ctx, d, 0, 1) for d in dev]
    budget = 4 * max(ibip.job_footprint(a.shape) for a in imgs)
    R = ibip.Router([0, 0], budget, max_slots=4)
    try:
        # nothing outstanding: the rule picks replica 0, then the other one
        assert R.route(imgs[0].shape) == (0, 0)
        tickets = [R.submit(torch.from_numpy(np.ascontiguousarray(a)), inlet=0, outlet=1) for a in imgs]
        res = [R.wait(t, timeout=600) for t in tickets]
        for r, a in zip(res, ref):
            assert r["status"] == 0 and r["K"] == a["K"]
            for k in ("seq", "step_r2", "step_centre", "trapped", "seq_out", "S", "Pc"):
                assert torch.equal(r[k], a[k]), k
        reps = [r["replica"] for r in res]
        assert reps[0] == 0 and reps[1] == 1   # the second request sees replica 0 busy
        st = [R.stats(k) for k in (0, 1)]
        assert st[0]["routed"] > 0 and st[1]["routed"] > 0
        assert st[0]["routed"] + st[1]["routed"] == len(imgs)
        assert st[0]["outstanding_voxels"] == 0 and st[1]["outstanding_voxels"] == 0
        assert st[0]["device"] == 0 and st[1]["device"] == 0
        # two results against the oracle itself
        for j in (0, 1):
            d = O.edt(imgs[j])
            s_ref = O.invade(imgs[j], d, inlet=0)[0]
            tr_ref, so_ref = O.trapping(s_ref, 1)
            assert np.array_equal(res[j]["seq"].cpu().numpy(), s_ref)
            assert np.array_equal(res[j]["seq_out"].cpu().numpy(), so_ref)
    finally:
        R.close()


def test_router_refuses_a_job_no_replica_holds(lib):
    ibip, ctx = lib
    R = ibip.Router([0], 1 << 20, max_slots=1)
    try:
        with pytest.raises(ibip.IbipError) as e:
            R.route((128, 128, 128))
        assert e.value.status == ibip.ERR_OOM
    finally:
        R.close()
