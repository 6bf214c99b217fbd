"""The widest path's work queue under contention: on small images most of
the persistent blocks wait for work, so a tile woken while it is being
relaxed is taken again at once by another block and two blocks relax it
together.  Trapping (Section 2.2.3) and the opening's trim (Section 2.4.1)
must still equal the oracle on every image; a stale relaxation that
lowered the field would leave voxels trapped or trimmed that are not."""
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


@pytest.mark.parametrize("block", range(4))
def test_queue_trapping_and_trim_many_small_images(ctx, block):
    rng = np.random.default_rng(4200 + block)
    for i in range(20):
        shape = tuple(int(x) for x in rng.integers(8, 56, 3))
        img = S.blobs(shape, rng.uniform(1.2, 3.0), rng.uniform(0.45, 0.75), rng) if i % 2 else \
            S.sphere_pack(shape, int(rng.integers(2, 6)), rng.uniform(0.3, 0.5), rng)
        inlet = int(rng.integers(0, 6))
        d = O.edt(img)
        seq = O.invade(img, d, inlet=inlet)[0]
        tr, so = ctx.trapping(torch.from_numpy(seq).cuda(), inlet ^ 1)
        rtr, rso = O.trapping(seq, inlet ^ 1)
        assert np.array_equal(tr.cpu().numpy(), rtr), (block, i, shape)
        assert np.array_equal(so.cpu().numpy(), rso), (block, i, shape)
        T = S.mio_levels(int(d[img > 0].max()) if img.any() else 1, 20)
        lev, cnt = ctx.morph_drainage(torch.from_numpy(img).cuda(), torch.from_numpy(d).cuda(), T, inlet=inlet)
        rlev, rcnt = O.morph_drainage(img, d, T, inlet=inlet)
        assert np.array_equal(lev.cpu().numpy(), rlev) and cnt == rcnt.tolist(), (block, i, shape)
