"""Shared-device mode (include/ibip.h, ibip_set_shared_device): the
widest-path propagation runs one ordinary launch per round instead of one
cooperative grid, so a context can run trapping and the opening's trim
beside a long kernel of another stream.  Results are the oracle's either
way: alone, and with the opening (Section 2.4.1) computed by a second
context on a low-priority stream from a worker thread while the first
context runs the invasion (Section 2.1), as the bench step does."""
import threading

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import ibip
    main, side = ibip.Context(0), ibip.Context(0)
    side.set_shared_device(True)
    return main, side


@pytest.mark.parametrize("seed", range(6))
def test_shared_device_trapping_and_opening(ctxs, seed):
    _, side = ctxs
    rng = np.random.default_rng(2100 + seed)
    shape = tuple(int(x) for x in rng.integers(8, 48, 3))
    img = S.blobs(shape, rng.uniform(1.5, 3.0), rng.uniform(0.5, 0.75), rng) if seed % 2 else \
        S.sphere_pack(shape, int(rng.integers(2, 5)), rng.uniform(0.35, 0.5), rng)
    d = O.edt(img)
    seq = O.invade(img, d, inlet=seed % 6)[0]
    tr, so = side.trapping(torch.from_numpy(seq).cuda(), seed % 6 ^ 1)
    rtr, rso = O.trapping(seq, seed % 6 ^ 1)
    assert np.array_equal(tr.cpu().numpy(), rtr) and np.array_equal(so.cpu().numpy(), rso)
    T = S.mio_levels(int(d[img > 0].max()) if img.any() else 1, 30)
    lev, cnt = side.morph_drainage(torch.from_numpy(img).cuda(), torch.from_numpy(d).cuda(), T, inlet=seed % 6)
    rlev, rcnt = O.morph_drainage(img, d, T, inlet=seed % 6)
    assert np.array_equal(lev.cpu().numpy(), rlev) and cnt == rcnt.tolist()


def test_opening_beside_a_running_invasion(ctxs):
    main, side = ctxs
    w = S.c2_spheres200()
    img = torch.from_numpy(w.image).cuda()
    d = main.edt(img)
    T = S.mio_levels(int(d[img > 0].max().item()), 40)
    hi = torch.cuda.Stream(priority=-1)
    lo = torch.cuda.Stream(priority=0)
    ready = torch.cuda.Event()
    ready.record()
    box = {}

    def opening():
        torch.cuda.set_device(0)
        lo.wait_event(ready)
        with torch.cuda.stream(lo):
            box["lev"], box["cnt"] = side.morph_drainage(img, d, T, inlet=0)

    t = threading.Thread(target=opening)
    with torch.cuda.stream(hi):
        hi.wait_event(ready)
        t.start()
        seq, r2, cen, K, st = main.invade(img, d, inlet=0)
        t.join()
        tr, so = main.trapping(seq, 1)
    torch.cuda.synchronize()
    dh = O.edt(w.image)
    rseq = O.invade(w.image, dh, inlet=0)[0]
    assert np.array_equal(seq.cpu().numpy(), rseq)
    assert np.array_equal(so.cpu().numpy(), O.trapping(rseq, 1)[1])
    rlev, rcnt = O.morph_drainage(w.image, dh, T, inlet=0)
    assert np.array_equal(box["lev"].cpu().numpy(), rlev) and box["cnt"] == rcnt.tolist()
