"""Plain CPU oracle for image-based invasion percolation (arXiv 2101.03240).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product library
never does.  The arithmetic lives in ``ibip_oracle.c`` (plain C, compiled
with gcc on first use); this module only marshals numpy arrays to it.

Functions mirror the C entry points; every array argument is a C-contiguous
numpy array with the image's shape (nx, ny, nz) unless stated otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibip_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
STEP_LIMIT = -4


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP) unless the shared object is newer
    than its source.  Returns the path of the shared object."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i32, i64, dbl = C.c_int, C.c_int64, C.c_double
            sig = {
                "or_edt_brute": (None, [P, i32, i32, i32, P]),
                "or_edt_sep": (None, [P, i32, i32, i32, P]),
                "or_invade_scan": (i64, [P, P, i32, i32, i32, i32, i64, P, P, P, i64, P]),
                "or_invade_heap": (i64, [P, P, i32, i32, i32, i32, i64, P, P, P, i64, P]),
                "or_invade_scan_mask": (i64, [P, P, i32, i32, i32, i32, P, i64, P, P, P, i64, P]),
                "or_invade_heap_mask": (i64, [P, P, i32, i32, i32, i32, P, i64, P, P, P, i64, P]),
                "or_invade_literal_scan": (i64, [P, P, i32, i32, i32, i32, i64, P, P, P, P, i64, P]),
                "or_invade_literal_queue": (i64, [P, P, i32, i32, i32, i32, i64, P, P, P, P, i64, P]),
                "or_trap_bfs": (None, [P, i32, i32, i32, i32, i32, P, P]),
                "or_trap_uf": (None, [P, i32, i32, i32, i32, i32, P, P]),
                "or_count_unconnected": (i64, [P, i32, i32, i32, i32]),
                "or_mio_plain": (None, [P, P, i32, i32, i32, i32, P, i32, P, P]),
                "or_mio_edt": (None, [P, P, i32, i32, i32, i32, P, i32, P, P]),
                "or_mio_plain_td": (None, [P, P, i32, i32, i32, i32, P, P, i32, P, P]),
                "or_mio_edt_td": (None, [P, P, i32, i32, i32, i32, P, P, i32, P, P]),
                "or_pc_curve": (None, [P, i64, P, i64, dbl, dbl, dbl, P, P, P]),
                "or_abi_version": (i32, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _img(image):
    a = np.ascontiguousarray(image, dtype=np.uint8)
    assert a.ndim == 3
    return a


def edt_brute(image):
    """Squared EDT by brute force over all solid voxels (Section 2.1)."""
    a = _img(image)
    out = np.empty(a.shape, np.int32)
    lib().or_edt_brute(_p(a), *a.shape, _p(out))
    return out


def edt(image):
    """Squared EDT by three separable 1-D min-plus passes (same values)."""
    a = _img(image)
    out = np.empty(a.shape, np.int32)
    lib().or_edt_sep(_p(a), *a.shape, _p(out))
    return out


def invade(image, dt2, inlet=0, max_steps=None, method="heap", capacity=None, mask=None):
    """Run the invasion (Section 2.1).  Returns (seq, step_r2, step_centre,
    status, K).  method: "heap" (priority queue) or "scan" (rescan every
    step).  mask: optional uint8 image of inlet voxels (nonzero), replacing
    the inlet face."""
    a = _img(image)
    d = np.ascontiguousarray(dt2, dtype=np.int32)
    n = a.size
    npore = int(np.count_nonzero(a))
    if max_steps is None:
        max_steps = npore
    cap = npore if capacity is None else int(capacity)
    seq = np.empty(a.shape, np.int32)
    r2 = np.zeros(max(cap, 1), np.int32)
    cen = np.zeros(max(cap, 1), np.int32)
    st = C.c_int(0)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    if m is not None and m.shape != a.shape:
        raise ValueError("mask shape differs from the image")
    f = lib().or_invade_heap_mask if method == "heap" else lib().or_invade_scan_mask
    k = f(_p(a), _p(d), *a.shape, int(inlet), None if m is None else _p(m), int(max_steps), _p(seq), _p(r2),
          _p(cen), cap, C.addressof(st))
    k = int(k)
    kk = min(k, cap)
    del n
    return seq, r2[:kk].copy(), cen[:kk].copy(), int(st.value), k


def invade_literal(image, dt2, inlet=0, max_steps=None, method="queue", capacity=None):
    """The invasion exactly as Section 2.1 prints it: candidates are the
    inlets plus their face neighbours, every candidate holding the largest
    value is an insertion point of the step, spheres have the truncated
    integer radius, insertion points join the inlets with their value set to
    zero.  Returns (seq, cstep, step_r2, step_count, status, K): cstep[v] is
    the step at which v was an insertion point (0 never), step_r2 the squared
    integer radius of each step, step_count its number of insertion points.
    method: "queue" (each voxel queued once) or "scan" (the definition)."""
    a = _img(image)
    d = np.ascontiguousarray(dt2, dtype=np.int32)
    npore = int(np.count_nonzero(a))
    if max_steps is None:
        max_steps = npore
    cap = npore if capacity is None else int(capacity)
    seq = np.empty(a.shape, np.int32)
    cstep = np.empty(a.shape, np.int32)
    r2 = np.zeros(max(cap, 1), np.int32)
    cnt = np.zeros(max(cap, 1), np.int32)
    st = C.c_int(0)
    f = lib().or_invade_literal_queue if method == "queue" else lib().or_invade_literal_scan
    k = int(f(_p(a), _p(d), *a.shape, int(inlet), int(max_steps), _p(seq), _p(cstep), _p(r2), _p(cnt), cap,
              C.addressof(st)))
    kk = min(k, cap)
    return seq, cstep, r2[:kk].copy(), cnt[:kk].copy(), int(st.value), k


def trapping(seq, outlet=1, rerank=False, method="uf"):
    """Defending-phase trapping (Section 2.2.3).  Returns (trapped uint8,
    seq_out int32)."""
    s = np.ascontiguousarray(seq, dtype=np.int32)
    tr = np.empty(s.shape, np.uint8)
    out = np.empty(s.shape, np.int32)
    f = lib().or_trap_uf if method == "uf" else lib().or_trap_bfs
    f(_p(s), *s.shape, int(outlet), int(bool(rerank)), _p(tr), _p(out))
    return tr, out


def count_unconnected(seq, inlet=0):
    """Invaded voxels not joined to the inlet face through voxels invaded no
    later than themselves (0 for a valid invasion)."""
    s = np.ascontiguousarray(seq, dtype=np.int32)
    return int(lib().or_count_unconnected(_p(s), *s.shape, int(inlet)))


def morph_drainage(image, dt2, levels, inlet=0, method="edt", dilate_levels=None):
    """Morphological-opening drainage (Section 2.4.1).  Level i erodes at
    dt2 >= levels[i] and dilates by the ball d^2 < dilate_levels[i] (default:
    the same bound).  Returns (level int32, counts int64[L])."""
    a = _img(image)
    d = np.ascontiguousarray(dt2, dtype=np.int32)
    T = np.ascontiguousarray(levels, dtype=np.int32)
    Td = T if dilate_levels is None else np.ascontiguousarray(dilate_levels, dtype=np.int32)
    assert Td.shape == T.shape
    lev = np.empty(a.shape, np.int32)
    cnt = np.zeros(max(len(T), 1), np.int64)
    f = lib().or_mio_edt_td if method == "edt" else lib().or_mio_plain_td
    f(_p(a), _p(d), *a.shape, int(inlet), _p(T), _p(Td), len(T), _p(lev), _p(cnt))
    return lev, cnt[:len(T)].copy()


def pc_curve(seq, step_r2, voxel_m=5e-6, sigma=0.072, theta_deg=180.0, sat_image=False):
    """Saturation and capillary pressure per step (Sections 2.2.1-2.2.2).
    Returns (S float32[K], Pc float32[K], sat_image float32 or None)."""
    s = np.ascontiguousarray(seq, dtype=np.int32)
    r2 = np.ascontiguousarray(step_r2, dtype=np.int32)
    K = len(r2)
    S = np.zeros(max(K, 1), np.float32)
    P = np.zeros(max(K, 1), np.float32)
    img = np.empty(s.shape, np.float32) if sat_image else None
    lib().or_pc_curve(_p(s), s.size, _p(r2), K, float(voxel_m), float(sigma), float(theta_deg),
                      _p(S), _p(P), _p(img))
    return S[:K].copy(), P[:K].copy(), img


def equal_saturation(seq, level, n_levels):
    """Equal-saturation comparison of an invasion with morphological-opening
    drainage (Section 3.1.1, Figure 8), by integer counts: for opening level
    i (0-based), n_i = voxels with 1 <= level <= i + 1; k_i = the smallest
    invasion step whose cumulative invaded count reaches n_i (the last step
    if none does); diff_i = size of the symmetric difference of
    {1 <= level <= i + 1} and {1 <= seq <= k_i}.  `level` uses the encoding
    of morph_drainage (-1 none, 0 solid, i + 1 first level).  Returns
    (k, diff, n) as int64 arrays of length n_levels."""
    s = np.asarray(seq).ravel()
    lv = np.asarray(level).ravel()
    K = int(s.max()) if s.size else 0
    K = max(K, 0)
    cum = np.cumsum(np.bincount(s[s >= 1], minlength=K + 1))   # cum[k] = voxels with 1 <= seq <= k
    ks, diffs, ns = [], [], []
    for i in range(n_levels):
        in_mio = (lv >= 1) & (lv <= i + 1)
        n = int(in_mio.sum())
        hit = np.nonzero(cum >= n)[0]
        k = int(hit[0]) if hit.size else K
        in_ibip = (s >= 1) & (s <= k)
        ks.append(k)
        ns.append(n)
        diffs.append(int(np.count_nonzero(in_mio != in_ibip)))
    return np.array(ks, np.int64), np.array(diffs, np.int64), np.array(ns, np.int64)


def pc_envelope(seq, step_r2, levels):
    """The drainage envelope of the invasion at the opening's pressures
    (Section 2.2.2 and Section 3.1.1: the envelope of the invasion's peak
    pressures is the opening's capillary-pressure curve).  Pc falls as the
    sphere radius grows, so the running peak of Pc up to step k is the Pc of
    the smallest step_r2 so far; at the opening's pressure of level i
    (squared radius levels[i]) the invasion has taken every step before its
    running-minimum r2 first drops below levels[i].  Returns (kstar, n):
    kstar[i] = that number of steps (the first step j with step_r2[j] <
    levels[i], minus one; K if none) and n[i] = voxels with
    1 <= seq <= kstar[i], as int64 arrays -- to be compared with the
    opening's cumulative counts at the same levels."""
    s = np.asarray(seq).ravel()
    r2 = np.asarray(step_r2, dtype=np.int64).ravel()
    K = r2.size
    cum = np.cumsum(np.bincount(s[(s >= 1) & (s <= K)], minlength=K + 1))   # cum[k] = voxels with 1 <= seq <= k
    ks, ns = [], []
    for T in levels:
        below = np.nonzero(r2 < int(T))[0]
        k = int(below[0]) if below.size else K    # steps 1..k all have r2 >= T
        ks.append(k)
        ns.append(int(cum[k]))
    return np.array(ks, np.int64), np.array(ns, np.int64)


def rerank_radii(seq, step_r2, outlet=1):
    """Trapping with re-ranking (Section 2.2.3) and the radii of the steps
    that keep at least one voxel, in their old order.  Returns (trapped,
    seq_out re-ranked, step_r2 of the surviving steps)."""
    tr, so = trapping(seq, outlet, rerank=False)
    kept = np.unique(so[so >= 1])
    r2 = np.asarray(step_r2)[kept - 1] if kept.size else np.zeros(0, np.int32)
    tr2, so2 = trapping(seq, outlet, rerank=True)
    return tr2, so2, np.asarray(r2, np.int32)


def size_image(seq, step_r2):
    """Squared radius of the sphere that invaded each voxel (Section 2.2.2,
    Figure 5 right): 0 on solid, -1 on uninvaded pore."""
    s = np.asarray(seq)
    r2 = np.asarray(step_r2)
    K = r2.size
    out = np.where(s == 0, 0, -1).astype(np.int32)
    inv = (s >= 1) & (s <= K)
    out[inv] = r2[s[inv] - 1]
    return out
