"""Parity at the full workload sizes, through the same entry points bench.py
times: the 200^3 sphere pack (the benchmark workload) and the 512^3
anisotropic blobs.  Integer outputs are compared element by element with
the oracle at every radius of the opening; at both sizes the opening's
oracle is its thresholded-EDT form, which the CPU tests hold bit-exact
with the plain ball-stamping definition."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def check_path(ctx, w, mio_exact_levels):
    img = w.image
    d_ref = O.edt(img)
    d = ctx.edt(dev(img))
    assert np.array_equal(host(d), d_ref)
    seq_ref, r2_ref, cen_ref, st_ref, K_ref = O.invade(img, d_ref, inlet=w.inlet)
    seq, r2, cen, K, st = ctx.invade(dev(img), d, inlet=w.inlet)
    assert K == K_ref and st == st_ref == 0
    assert np.array_equal(host(seq), seq_ref)
    assert np.array_equal(host(r2), r2_ref) and np.array_equal(host(cen), cen_ref)
    tr_ref, so_ref = O.trapping(seq_ref, w.outlet)
    tr, so = ctx.trapping(seq, w.outlet)
    assert np.array_equal(host(tr), tr_ref) and np.array_equal(host(so), so_ref)
    Sr, Pr, _ = O.pc_curve(so_ref, r2_ref, w.voxel_m, w.sigma, w.theta_deg)
    Sg, Pg, _ = ctx.pc_curve(so, r2, w.voxel_m, w.sigma, w.theta_deg)
    assert np.array_equal(host(Sg), Sr) and np.array_equal(host(Pg), Pr)
    # opening at the 40 radii of the workload
    T = S.mio_levels(int(d_ref[img == 1].max()), 40)
    lev, cnt = ctx.morph_drainage(dev(img), d, T, inlet=w.inlet)
    lev = host(lev)
    assert (np.diff(cnt) >= 0).all()
    assert ((lev == 0) == (img == 0)).all()
    k = len(T) if mio_exact_levels is None else mio_exact_levels
    lev_ref, cnt_ref = O.morph_drainage(img, d_ref, T[:k], inlet=w.inlet,
                                        method="edt" if mio_exact_levels is None else "plain")
    assert np.array_equal(np.where(lev > k, -1, lev), lev_ref)
    assert cnt[:k] == cnt_ref.tolist()
    return seq_ref, so_ref, lev, cnt, T


def test_full_spheres200(ctx):
    """The benchmark workload, every output bit for bit (all 39 radii)."""
    check_path(ctx, S.c2_spheres200(), None)


def test_full_blobs512(ctx):
    """512^3 blobs (sigma 4,8,4, porosity 0.6): EDT, 5 M-step invasion,
    trapping, Pc and the opening at all of its radii, bit for bit."""
    w = S.c3_blobs512()
    seq_ref, so_ref, lev, cnt, T = check_path(ctx, w, None)
    assert cnt[-1] > 0
    # every opened voxel is pore and was reachable by the invasion
    assert ((lev >= 1) <= (seq_ref >= 1)).all()
