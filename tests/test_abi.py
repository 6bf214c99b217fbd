"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point include/ibip.h declares, and
rejects bad arguments before touching the device.  Also checks that the
oracle and the CUDA sources share nothing."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_03240_gb300 import build_lib
    path = build_lib.build()
    return C.CDLL(path)


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ibip.h")).read()
    return re.findall(r"IBIP_API\s+[\w\s\*]+?\b(ibip_\w+)\s*\(", txt)


def test_header_declares_the_calls():
    names = set(declared_symbols())
    for n in ["ibip_create", "ibip_destroy", "ibip_edt", "ibip_invade", "ibip_trapping",
              "ibip_morph_drainage", "ibip_pc_curve", "ibip_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_status_strings(lib):
    f = lib.ibip_status_string
    f.restype = C.c_char_p
    f.argtypes = [C.c_int]
    assert f(0) == b"ok"
    assert b"argument" in f(-1)
    assert b"step limit" in f(-4)


def test_null_arguments_rejected_on_host(lib):
    class Dims(C.Structure):
        _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]
    lib.ibip_edt.argtypes = [C.c_void_p, C.c_void_p, Dims, C.c_void_p]
    assert lib.ibip_edt(None, None, Dims(4, 4, 4), None) == -1
    lib.ibip_create.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    assert lib.ibip_create(None, 0, None) == -1
    lib.ibip_destroy.argtypes = [C.c_void_p]
    assert lib.ibip_destroy(None) == -1
    lib.ibip_get_stream.argtypes = [C.c_void_p, C.c_void_p]
    out = C.c_void_p()
    assert lib.ibip_get_stream(None, C.byref(out)) == -1
    lib.ibip_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.ibip_set_stream(None, None) == -1
    lib.ibip_set_shared_device.argtypes = [C.c_void_p, C.c_int]
    assert lib.ibip_set_shared_device(None, 1) == -1


def test_oracle_and_cuda_path_share_nothing():
    csrc = os.path.join(ROOT, "paper_2101_03240_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower() or f.endswith(".md"), f
    otxt = open(os.path.join(ROOT, "oracle", "ibip_oracle.c")).read()
    assert "#include \"" not in otxt and "csrc" not in otxt and "ibip.h" not in otxt
    for f in ("ibip.py", "build_lib.py", "synth.py", "__init__.py"):
        txt = open(os.path.join(ROOT, "paper_2101_03240_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_checked_build_compiles_and_exports_every_symbol(lib):
    """The bounds-checked build (IBIP_CHECKED=1) is a separate library in
    _build_checked/; it must keep compiling and export the same calls."""
    import subprocess
    import sys
    env = dict(os.environ, IBIP_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "from paper_2101_03240_gb300 import build_lib; print(build_lib.build())"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    path = r.stdout.strip().splitlines()[-1]
    assert "_build_checked" in path and os.path.exists(path)
    checked = C.CDLL(path)
    for n in declared_symbols():
        assert hasattr(checked, n), n
