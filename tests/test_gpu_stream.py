"""The context's stream (include/ibip.h, ibip_create / ibip_set_stream /
ibip_get_stream), called through the C ABI: with no stream given a context
queues on a non-blocking stream of its own; the legacy default stream is
used only when asked for by its explicit handle; NULL in ibip_set_stream
returns to the context's own stream.  Each stream choice computes the same
squared EDT as the oracle."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LEGACY, PER_THREAD = 1, 2


class Dims(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import build_lib
    L = C.CDLL(build_lib.LIB)
    L.ibip_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]
    L.ibip_destroy.argtypes = [C.c_void_p]
    L.ibip_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.ibip_get_stream.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
    L.ibip_edt.argtypes = [C.c_void_p, C.c_void_p, Dims, C.c_void_p]
    L.ibip_synchronize.argtypes = [C.c_void_p]
    return L


def stream_of(L, h):
    s = C.c_void_p()
    assert L.ibip_get_stream(h, C.byref(s)) == 0
    return s.value or 0


def edt_on(L, h, img):
    d = torch.from_numpy(img).cuda()
    out = torch.full(img.shape, -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert L.ibip_edt(h, C.c_void_p(d.data_ptr()), Dims(*img.shape), C.c_void_p(out.data_ptr())) == 0
    assert L.ibip_synchronize(h) == 0
    return out.cpu().numpy()


def test_default_is_an_own_stream_and_legacy_is_explicit(lib):
    torch.cuda.set_device(0)
    rng = np.random.default_rng(77)
    img = S.blobs((40, 33, 29), 2.0, 0.6, rng)
    want = O.edt(img)
    h = C.c_void_p()
    assert lib.ibip_create(C.byref(h), 0, None) == 0
    try:
        own = stream_of(lib, h)
        assert own not in (0, LEGACY, PER_THREAD)
        assert np.array_equal(edt_on(lib, h, img), want)
        # the legacy default stream, given by its handle, then back to the own one
        assert lib.ibip_set_stream(h, C.c_void_p(LEGACY)) == 0
        assert stream_of(lib, h) == LEGACY
        assert np.array_equal(edt_on(lib, h, img), want)
        assert lib.ibip_set_stream(h, None) == 0
        assert stream_of(lib, h) == own
        assert np.array_equal(edt_on(lib, h, img), want)
    finally:
        assert lib.ibip_destroy(h) == 0


def test_caller_stream_and_legacy_at_creation(lib):
    torch.cuda.set_device(0)
    rng = np.random.default_rng(78)
    img = S.sphere_pack((36, 30, 41), 4, 0.45, rng)
    want = O.edt(img)
    for given in (LEGACY, PER_THREAD):
        h = C.c_void_p()
        assert lib.ibip_create(C.byref(h), 0, C.c_void_p(given)) == 0
        try:
            assert stream_of(lib, h) == given
            assert np.array_equal(edt_on(lib, h, img), want)
            # NULL later: a stream of the context's own is created on demand
            assert lib.ibip_set_stream(h, None) == 0
            assert stream_of(lib, h) not in (0, LEGACY, PER_THREAD)
            assert np.array_equal(edt_on(lib, h, img), want)
        finally:
            assert lib.ibip_destroy(h) == 0
    s = torch.cuda.Stream()
    h = C.c_void_p()
    assert lib.ibip_create(C.byref(h), 0, C.c_void_p(s.cuda_stream)) == 0
    try:
        assert stream_of(lib, h) == s.cuda_stream
        assert np.array_equal(edt_on(lib, h, img), want)
    finally:
        assert lib.ibip_destroy(h) == 0
