"""Cancellation of the invasion (ibip_cancel) and host-side fault injection
(ibip_debug_fail_alloc).  Nothing here faults or hangs the GPU: the kernel
reads a host-mapped flag and returns a status, and the injected failure is
a refused scratch allocation on the host.  After each, the context must
still give the oracle's results."""
import threading
import time

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ibip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import ibip as m
    return m


@pytest.fixture(scope="module")
def spheres():
    """The 200^3 sphere pack: its invasion runs ~0.2 s on the GPU."""
    img = S.c2_spheres200().image
    return img, torch.from_numpy(img).cuda()


def _prefix(seq_full, k):
    """The sequence image of the first k steps of a full run."""
    s = seq_full.copy()
    s[(s > k)] = -1
    return s


def test_cancel_before_start_stops_at_step_zero(ibip):
    rng = np.random.default_rng(3)
    img = S.blobs((30, 28, 26), 2.0, 0.6, rng)
    d_img = torch.from_numpy(img).cuda()
    ctx = ibip.Context(0)
    d = ctx.edt(d_img)
    ctx.cancel(True)
    seq, r2, cen, K, st = ctx.invade(d_img, d, check=False)
    assert st == ibip.ERR_CANCELLED and K == 0
    assert np.array_equal(seq.cpu().numpy(), np.where(img > 0, -1, 0).astype(np.int32))
    # the request was served: the next call runs to the end
    seq, r2, cen, K, st = ctx.invade(d_img, d)
    s_ref, r2_ref, c_ref, st_ref, K_ref = O.invade(img, O.edt(img), inlet=0)
    assert st == ibip.OK and K == K_ref and np.array_equal(seq.cpu().numpy(), s_ref)


def test_withdrawn_request_does_not_cancel(ibip):
    rng = np.random.default_rng(4)
    img = S.blobs((24, 30, 22), 2.0, 0.6, rng)
    d_img = torch.from_numpy(img).cuda()
    ctx = ibip.Context(0)
    ctx.cancel(True)
    ctx.cancel(False)
    seq, r2, cen, K, st = ctx.invade(d_img)
    assert st == ibip.OK
    assert np.array_equal(seq.cpu().numpy(), O.invade(img, O.edt(img), inlet=0)[0])
    assert ibip._lib().ibip_cancel(ctx._h, 2) == ibip.ERR_ARG
    assert ibip._lib().ibip_cancel(None, 1) == ibip.ERR_ARG


def test_cancel_mid_run_leaves_a_prefix_that_resumes_exactly(ibip, spheres):
    img, d_img = spheres
    ctx = ibip.Context(0)
    d = ctx.edt(d_img)
    seq_f, r2_f, cen_f, K_f, st_f = ctx.invade(d_img, d)   # also warms every scratch slot
    seq_f, r2_f, cen_f = seq_f.cpu().numpy(), r2_f.cpu().numpy(), cen_f.cpu().numpy()
    assert st_f == ibip.OK and K_f > 1000
    out = {}

    def run():
        out["r"] = ctx.invade(d_img, d, check=False)

    # the invasion takes ~0.2 s; if a slow thread start lets it finish before
    # the request arrives, try again with a shorter delay (a request that
    # arrives before the first flag read stops it at K = 0, also valid)
    for delay in (0.06, 0.03, 0.01, 0.0):
        t = threading.Thread(target=run)
        t.start()
        time.sleep(delay)
        ctx.cancel(True)
        t.join(timeout=120)
        assert not t.is_alive()
        seq, r2, cen, K, st = out["r"]
        if st == ibip.ERR_CANCELLED:
            break
        assert st == ibip.OK and K == K_f   # finished first: the flag is still set
        ctx.cancel(False)
    assert st == ibip.ERR_CANCELLED, st
    assert 0 <= K < K_f
    assert np.array_equal(seq.cpu().numpy(), _prefix(seq_f, K))
    assert np.array_equal(r2.cpu().numpy(), r2_f[:K]) and np.array_equal(cen.cpu().numpy(), cen_f[:K])
    # resuming the cancelled run gives the uninterrupted result
    seq2, r22, cen2, K2, st2 = ctx.invade_ex(d_img, d, resume_from=(seq, r2, cen))
    assert st2 == ibip.OK and K2 == K_f
    assert np.array_equal(seq2.cpu().numpy(), seq_f)
    assert np.array_equal(r22.cpu().numpy(), r2_f) and np.array_equal(cen2.cpu().numpy(), cen_f)


def test_cancel_stops_every_image_of_a_batch(ibip):
    rng = np.random.default_rng(8)
    imgs = [S.blobs((20 + 3 * i, 22, 18), 2.0, 0.6, rng) for i in range(4)]
    dev = [torch.from_numpy(a).cuda() for a in imgs]
    ctx = ibip.Context(0)
    ctx.cancel(True)
    res = ctx.invade_batched(dev, 0, trapping=False, curve=False, check=False)
    assert all(r["status"] == ibip.ERR_CANCELLED and r["K"] == 0 for r in res)
    res = ctx.invade_batched(dev, 0, trapping=False, curve=False)
    for a, r in zip(imgs, res):
        assert r["status"] == ibip.OK
        assert np.array_equal(r["seq"].cpu().numpy(), O.invade(a, O.edt(a), inlet=0)[0])


@pytest.mark.parametrize("nth", [1, 2, 3, 5])
def test_injected_allocation_failure_then_recovery(ibip, nth):
    rng = np.random.default_rng(10 + nth)
    img = S.sphere_pack((34, 30, 38), 3, 0.45, rng)
    d_img = torch.from_numpy(img).cuda()
    ctx = ibip.Context(0)             # fresh: every scratch slot must be allocated
    ctx.debug_fail_alloc(nth)
    with pytest.raises(ibip.IbipError) as e:
        for _ in range(3):            # the nth allocation falls in one of these calls
            d = ctx.edt(d_img)
            ctx.invade(d_img, d)
            ctx.trapping(ctx.invade(d_img, d)[0], 1)
    assert e.value.status == ibip.ERR_OOM
    # the context recovers: allocations succeed again and results are exact
    d = ctx.edt(d_img)
    dref = O.edt(img)
    assert np.array_equal(d.cpu().numpy(), dref)
    seq, r2, cen, K, st = ctx.invade(d_img, d)
    s_ref = O.invade(img, dref, inlet=0)[0]
    assert st == ibip.OK and np.array_equal(seq.cpu().numpy(), s_ref)
    tr, so = ctx.trapping(seq, 1)
    tr_ref, so_ref = O.trapping(s_ref, 1)
    assert np.array_equal(tr.cpu().numpy(), tr_ref) and np.array_equal(so.cpu().numpy(), so_ref)
    with pytest.raises(ibip.IbipError):
        ctx.debug_fail_alloc(-1)
