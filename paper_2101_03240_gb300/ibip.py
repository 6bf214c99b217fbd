"""Thin ctypes binding over libibip (include/ibip.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Tensors are PyTorch CUDA tensors (PyTorch provides device memory and
streams); work is queued on the current PyTorch stream.  If the library is
missing this module raises at import of the first call -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

# CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware work queues
# (8 unless set).  A server runs many slots, each with two streams; when
# they outnumber the queues, a slot's long one-CTA invasion kernel holds up
# every later launch of the other streams sharing its queue (small requests
# then wait for seconds behind a large one).  32 is the largest value; it
# only takes effect if set before the process creates its CUDA context, and
# a value the user set is kept.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import torch  # noqa: E402

from . import build_lib

OK = 0
ERR_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_STEP_LIMIT = -4
ERR_NOT_CONVERGED = -5
ERR_CANCELLED = -6

# cudaStreamLegacy: the explicit handle of CUDA's legacy default stream
CUDA_STREAM_LEGACY = 1

FACES = {"x0": 0, "x1": 1, "y0": 2, "y1": 3, "z0": 4, "z1": 5}


class Dims(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class Job(C.Structure):
    _fields_ = [("image", C.c_void_p), ("dims", Dims), ("inlet", C.c_int32), ("outlet", C.c_int32),
                ("dt2", C.c_void_p), ("seq", C.c_void_p), ("step_r2", C.c_void_p), ("step_centre", C.c_void_p),
                ("capacity_steps", C.c_int64), ("trapped", C.c_void_p), ("seq_out", C.c_void_p),
                ("sat_per_step", C.c_void_p), ("pc_per_step", C.c_void_p), ("voxel_m", C.c_double),
                ("sigma", C.c_double), ("theta_deg", C.c_double), ("n_steps", C.c_int64), ("status", C.c_int32)]


class LiteralJob(C.Structure):
    _fields_ = [("image", C.c_void_p), ("dims", Dims), ("inlet", C.c_int32), ("dt2", C.c_void_p),
                ("max_steps", C.c_int64), ("seq", C.c_void_p), ("cstep", C.c_void_p), ("step_r2", C.c_void_p),
                ("step_count", C.c_void_p), ("capacity_steps", C.c_int64), ("n_steps", C.c_int64),
                ("status", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("slot", C.c_int32), ("n_steps", C.c_int64), ("t_submit_ns", C.c_int64),
                ("t_start_ns", C.c_int64), ("t_end_ns", C.c_int64), ("mem_reserved", C.c_int64),
                ("mem_used", C.c_int64)]


class IbipError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        msg = _lib().ibip_status_string(status).decode()
        super().__init__("%s failed: %s (%d)" % (fn, msg, status))


_L = None
_lock = threading.Lock()


def lib_path() -> str:
    return build_lib.LIB


def _lib():
    global _L
    with _lock:
        if _L is None:
            if not os.path.exists(build_lib.LIB):
                raise RuntimeError("libibip.so is not built (%s); run __graft_entry__.build()" % build_lib.LIB)
            L = C.CDLL(build_lib.LIB)
            P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            sig = {
                "ibip_create": (C.c_int, [C.POINTER(P), C.c_int, P]),
                "ibip_destroy": (C.c_int, [P]),
                "ibip_set_stream": (C.c_int, [P, P]),
                "ibip_get_stream": (C.c_int, [P, C.POINTER(P)]),
                "ibip_edt": (C.c_int, [P, P, Dims, P]),
                "ibip_invade": (C.c_int, [P, P, P, Dims, C.c_int, i64, P, P, P, i64, C.POINTER(i64)]),
                "ibip_trapping": (C.c_int, [P, P, Dims, C.c_int, C.c_int, P, P]),
                "ibip_morph_drainage": (C.c_int, [P, P, P, Dims, C.c_int, P, i32, P, P]),
                "ibip_morph_drainage_ex": (C.c_int, [P, P, P, Dims, C.c_int, P, P, i32, P, P]),
                "ibip_pc_curve": (C.c_int, [P, P, Dims, P, i64, dbl, dbl, dbl, P, P, P]),
                "ibip_synchronize": (C.c_int, [P]),
                "ibip_launch_count": (i64, [P]),
                "ibip_status_string": (C.c_char_p, [C.c_int]),
                "ibip_profile_enable": (C.c_int, [P, C.c_int]),
                "ibip_invade_batched": (C.c_int, [P, i32, P]),
                "ibip_invade_stats": (C.c_int, [P, C.POINTER(i64), C.c_int]),
                "ibip_invade_trace": (C.c_int, [P, P, i64]),
                "ibip_set_autotune": (C.c_int, [P, C.c_int, C.c_char_p]),
                "ibip_cancel": (C.c_int, [P, C.c_int]),
                "ibip_debug_fail_alloc": (C.c_int, [P, C.c_int]),
                "ibip_set_edt_tiles": (C.c_int, [P, C.c_int, C.c_int]),
                "ibip_edt_tiles": (C.c_int, [P, Dims, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "ibip_profile_read": (C.c_int, [P, C.c_int, C.POINTER(dbl), C.POINTER(i64)]),
                "ibip_job_footprint": (i64, [Dims, C.c_int]),
                "ibip_trapping_ex": (C.c_int, [P, P, Dims, C.c_int, P, P, P, i64, P, C.POINTER(i64)]),
                "ibip_size_image": (C.c_int, [P, P, Dims, P, i64, P]),
                "ibip_invade_ex": (C.c_int, [P, P, P, Dims, C.c_int, P, C.c_int, i64, P, P, P, i64, C.POINTER(i64)]),
                "ibip_equal_saturation": (C.c_int, [P, P, P, Dims, i64, i32, C.POINTER(i64), C.POINTER(i64),
                                                    C.POINTER(i64)]),
                "ibip_invade_literal": (C.c_int, [P, P, P, Dims, C.c_int, i64, P, P, P, P, i64, C.POINTER(i64)]),
                "ibip_server_create": (C.c_int, [C.POINTER(P), P, C.c_size_t, C.c_int]),
                "ibip_server_destroy": (C.c_int, [P]),
                "ibip_server_submit": (C.c_int, [P, C.POINTER(Job), C.POINTER(C.c_uint64)]),
                "ibip_server_poll": (C.c_int, [P, C.c_uint64, C.POINTER(C.c_int), C.POINTER(Result)]),
                "ibip_server_wait": (C.c_int, [P, C.c_uint64, i64, C.POINTER(C.c_int), C.POINTER(Result)]),
                "ibip_server_stats": (C.c_int, [P, C.POINTER(i64), C.c_int]),
                "ibip_route_pick": (C.c_int, [C.c_int, C.POINTER(i64), C.POINTER(i64), i64]),
                "ibip_invade_literal_batched": (C.c_int, [P, i32, P, C.POINTER(C.c_int)]),
                "ibip_set_literal_cluster": (C.c_int, [P, C.c_int]),
                "ibip_set_shared_device": (C.c_int, [P, C.c_int]),
                "ibip_pc_envelope": (C.c_int, [P, P, Dims, P, i64, P, i32, C.POINTER(i64), C.POINTER(i64)]),
                "ibip_router_create": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int), C.c_size_t, C.c_int]),
                "ibip_router_destroy": (C.c_int, [P]),
                "ibip_router_route": (C.c_int, [P, Dims, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "ibip_router_submit": (C.c_int, [P, C.c_int, C.POINTER(Job), C.POINTER(C.c_uint64)]),
                "ibip_router_wait": (C.c_int, [P, C.c_uint64, i64, C.POINTER(C.c_int), C.POINTER(Result),
                                               C.POINTER(C.c_int)]),
                "ibip_router_stats": (C.c_int, [P, C.c_int, C.POINTER(i64), C.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _L = L
    return _L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dims(shape):
    nx, ny, nz = (int(s) for s in shape)
    return Dims(nx, ny, nz)


def _need(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.dim() == 3):
        raise ValueError("%s must be a contiguous 3-D CUDA %s tensor" % (name, dtype))


def _fill_job(J, im, inlet, outlet, trapping, curve, voxel_m, sigma, theta_deg):
    """Allocates the outputs of one image and fills its ibip_job."""
    _need(im, torch.uint8, "image")
    dev, N = im.device, im.numel()
    r = {"seq": torch.empty(im.shape, dtype=torch.int32, device=dev),
         "step_r2": torch.empty(max(N, 1), dtype=torch.int32, device=dev),
         "step_centre": torch.empty(max(N, 1), dtype=torch.int32, device=dev)}
    if trapping:
        r["trapped"] = torch.empty(im.shape, dtype=torch.uint8, device=dev)
        r["seq_out"] = torch.empty(im.shape, dtype=torch.int32, device=dev)
    if curve:
        r["S"] = torch.empty(max(N, 1), dtype=torch.float32, device=dev)
        r["Pc"] = torch.empty(max(N, 1), dtype=torch.float32, device=dev)
    J.image = im.data_ptr()
    J.dims = _dims(im.shape)
    J.inlet, J.outlet = inlet, outlet if trapping else -1
    J.dt2 = None
    J.seq, J.step_r2, J.step_centre = r["seq"].data_ptr(), r["step_r2"].data_ptr(), r["step_centre"].data_ptr()
    J.capacity_steps = N
    J.trapped = r["trapped"].data_ptr() if trapping else None
    J.seq_out = r["seq_out"].data_ptr() if trapping else None
    J.sat_per_step = r["S"].data_ptr() if curve else None
    J.pc_per_step = r["Pc"].data_ptr() if curve else None
    J.voxel_m, J.sigma, J.theta_deg = float(voxel_m), float(sigma), float(theta_deg)
    return r


def _trim(r, K):
    for key in ("step_r2", "step_centre", "S", "Pc"):
        if key in r:
            r[key] = r[key][:K]
    return r


def job_footprint(shape, with_dt2=True) -> int:
    """Upper bound of the device scratch bytes one served job of this shape
    takes (ibip_job_footprint)."""
    return int(_lib().ibip_job_footprint(_dims(shape), 1 if with_dt2 else 0))


class Context:
    """One libibip context on a CUDA device; calls queue on the current
    PyTorch stream of that device."""

    def __init__(self, device=None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device) \
            if not isinstance(device, torch.device) else device
        self.device = dev
        h = C.c_void_p()
        st = _lib().ibip_create(C.byref(h), dev.index, None)
        if st != OK:
            raise IbipError("ibip_create", st)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().ibip_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        # PyTorch's default stream has handle 0, the legacy default stream;
        # the ABI reads NULL as the context's own stream, so pass the legacy
        # stream's explicit handle instead
        s = torch.cuda.current_stream(self.device)
        _lib().ibip_set_stream(self._h, C.c_void_p(s.cuda_stream or CUDA_STREAM_LEGACY))

    @property
    def launches(self) -> int:
        return int(_lib().ibip_launch_count(self._h))

    def profile(self, on: bool):
        """Per-kernel-class CUDA-event timing on (clears the log) or off."""
        st = _lib().ibip_profile_enable(self._h, int(bool(on)))
        if st != OK:
            raise IbipError("ibip_profile_enable", st)

    def profile_read(self, cls: int):
        """(summed milliseconds, number of spans) of a kernel class since
        profiling was turned on (classes: see ibip_kernel_class)."""
        ms, n = C.c_double(0), C.c_int64(0)
        st = _lib().ibip_profile_read(self._h, int(cls), C.byref(ms), C.byref(n))
        if st != OK:
            raise IbipError("ibip_profile_read", st)
        return float(ms.value), int(n.value)

    def invade_stats(self) -> dict:
        """Counters of the last invade call (see ibip_invade_stats)."""
        a = (C.c_int64 * 48)()
        _lib().ibip_invade_stats(self._h, a, 48)
        keys = ["steps", "status", "iterations", "cycles_select", "cycles_bound", "cycles_commit", "items",
                "items_committed", "stale_bits", "rows_committed", "cycles_small_batches", "small_batches",
                "sel_gather", "sel_items", "sel_pairs", "sel_tail", "small_select", "small_bound", "small_commit",
                "tiny_iterations", "tiny_steps", "cycles_tiny", "s3_cont", "s3_prefix", "bound_list",
                "bound_ranks", "commit_stamp", "commit_queue", "tiny_gather", "tiny_bound", "mm_rounds",
                "mm_activations", "mm_sweeps", "tiny_commit", "bounds_violations", "first_unit_rank", "trace_batches",
                "span_cycles", "span_ns", "shell_units", "shell_listed", "removed", "single_batches",
                "tiny_merged", "tiny_merge_cycles", "gather_rounds", "gathers"]
        return dict(zip(keys, [int(x) for x in a]))

    def cancel(self, on: bool = True):
        """Request (or withdraw) cancellation of this context's invasion
        (see ibip_cancel); callable from another thread."""
        st = _lib().ibip_cancel(self._h, int(bool(on)))
        if st != OK:
            raise IbipError("ibip_cancel", st)

    def debug_fail_alloc(self, nth: int):
        """Test hook: fail the nth scratch allocation from now (0: off)."""
        st = _lib().ibip_debug_fail_alloc(self._h, int(nth))
        if st != OK:
            raise IbipError("ibip_debug_fail_alloc", st)

    def set_autotune(self, on: bool, cache_path: str | None = None):
        """Tile-shape autotuning of the EDT (see ibip_set_autotune)."""
        st = _lib().ibip_set_autotune(self._h, int(bool(on)), None if cache_path is None else cache_path.encode())
        if st != OK:
            raise IbipError("ibip_set_autotune", st)

    def set_edt_tiles(self, z_warps: int, strip_warps: int):
        """Force an EDT tile shape ((0, 0): automatic)."""
        st = _lib().ibip_set_edt_tiles(self._h, int(z_warps), int(strip_warps))
        if st != OK:
            raise IbipError("ibip_set_edt_tiles", st)

    def edt_tiles(self, shape) -> tuple:
        """(z_warps, strip_warps) an EDT of this shape would use now."""
        zw, sw = C.c_int(0), C.c_int(0)
        st = _lib().ibip_edt_tiles(self._h, _dims(shape), C.byref(zw), C.byref(sw))
        if st != OK:
            raise IbipError("ibip_edt_tiles", st)
        return int(zw.value), int(sw.value)

    def invade_trace(self, buf):
        """Record one row per batch of later invade calls into `buf` (CUDA
        int32 tensor of shape (n, 8): first step, steps, SM cycles, loop,
        items, rows stamped, shell rows, shell candidates), or stop
        recording (None).  See ibip_invade_trace."""
        if buf is None:
            st = _lib().ibip_invade_trace(self._h, None, 0)
        else:
            assert buf.is_cuda and buf.dtype == torch.int32 and buf.dim() == 2 and buf.shape[1] == 8
            assert buf.is_contiguous()
            st = _lib().ibip_invade_trace(self._h, _ptr(buf), buf.shape[0])
        if st != OK:
            raise IbipError("ibip_invade_trace", st)
        self._trace = buf

    def synchronize(self):
        st = _lib().ibip_synchronize(self._h)
        if st != OK:
            raise IbipError("ibip_synchronize", st)

    # -- calls ------------------------------------------------------------
    def edt(self, image, out=None):
        """Squared EDT of the pore space (int32)."""
        _need(image, torch.uint8, "image")
        out = torch.empty(image.shape, dtype=torch.int32, device=image.device) if out is None else out
        self._stream()
        st = _lib().ibip_edt(self._h, _ptr(image), _dims(image.shape), _ptr(out))
        if st != OK:
            raise IbipError("ibip_edt", st)
        return out

    def invade(self, image, dt2=None, inlet=0, max_steps=None, capacity=None, centres=True, seq=None,
               step_r2=None, step_centre=None, check=True):
        """Invasion sequence.  Returns (seq, step_r2[:K], step_centre[:K] or
        None, K, status)."""
        _need(image, torch.uint8, "image")
        if dt2 is not None:
            _need(dt2, torch.int32, "dt2")
        n = image.numel()
        if capacity is None:
            capacity = n if step_r2 is None else step_r2.numel()
        if max_steps is None:
            max_steps = n
        dev = image.device
        seq = torch.empty(image.shape, dtype=torch.int32, device=dev) if seq is None else seq
        step_r2 = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev) if step_r2 is None else step_r2
        if centres and step_centre is None:
            step_centre = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
        K = C.c_int64(0)
        self._stream()
        st = _lib().ibip_invade(self._h, _ptr(image), _ptr(dt2), _dims(image.shape), int(inlet), int(max_steps),
                                _ptr(seq), _ptr(step_r2), _ptr(step_centre) if centres else None, int(capacity),
                                C.byref(K))
        if check and st not in (OK, ERR_STEP_LIMIT):
            raise IbipError("ibip_invade", st)
        k = int(K.value)
        kk = min(k, capacity)
        return seq, step_r2[:kk], (step_centre[:kk] if centres else None), k, st

    def invade_ex(self, image, dt2=None, inlet=0, inlet_mask=None, resume_from=None, max_steps=None,
                  capacity=None):
        """ibip_invade_ex: `inlet_mask` (uint8 CUDA tensor, nonzero = inlet
        voxels) replaces the inlet face; `resume_from` = (seq, step_r2,
        step_centre) of an earlier call continues that run (the tensors are
        updated in place).  Returns (seq, step_r2, step_centre, K, status)
        with the step arrays trimmed to K."""
        _need(image, torch.uint8, "image")
        if dt2 is not None:
            _need(dt2, torch.int32, "dt2")
        if inlet_mask is not None:
            _need(inlet_mask, torch.uint8, "inlet_mask")
        dev, N = image.device, image.numel()
        cap = N if capacity is None else int(capacity)
        if resume_from is not None:
            seq, r2p, cp = resume_from
            r2 = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            cen = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            r2[:r2p.numel()] = r2p
            cen[:cp.numel()] = cp
        else:
            seq = torch.empty(image.shape, dtype=torch.int32, device=dev)
            r2 = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            cen = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        k = C.c_int64(0)
        self._stream()
        st = _lib().ibip_invade_ex(self._h, _ptr(image), _ptr(dt2), _dims(image.shape), int(inlet), _ptr(inlet_mask),
                                   1 if resume_from is not None else 0, N if max_steps is None else int(max_steps),
                                   _ptr(seq), _ptr(r2), _ptr(cen), cap, C.byref(k))
        if st not in (OK, ERR_STEP_LIMIT):
            raise IbipError("ibip_invade_ex", st)
        K = int(k.value)
        return seq, r2[:min(K, cap)], cen[:min(K, cap)], K, st

    def invade_literal(self, image, dt2=None, inlet=0, max_steps=None, capacity=None):
        """The invasion exactly as Section 2.1 prints it (ibip_invade_literal).
        Returns (seq, cstep, step_r2, step_count, K, status)."""
        _need(image, torch.uint8, "image")
        if dt2 is not None:
            _need(dt2, torch.int32, "dt2")
        dev, N = image.device, image.numel()
        cap = N if capacity is None else int(capacity)
        seq = torch.empty(image.shape, dtype=torch.int32, device=dev)
        cstep = torch.empty(image.shape, dtype=torch.int32, device=dev)
        r2 = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        cnt = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        k = C.c_int64(0)
        self._stream()
        st = _lib().ibip_invade_literal(self._h, _ptr(image), _ptr(dt2), _dims(image.shape), int(inlet),
                                        N if max_steps is None else int(max_steps), _ptr(seq), _ptr(cstep),
                                        _ptr(r2), _ptr(cnt), cap, C.byref(k))
        if st not in (OK, ERR_STEP_LIMIT):
            raise IbipError("ibip_invade_literal", st)
        K = int(k.value)
        return seq, cstep, r2[:min(K, cap)], cnt[:min(K, cap)], K, st

    def set_shared_device(self, on: bool):
        """Let this context's kernels run beside long-running kernels of
        other streams (ibip_set_shared_device): the widest-path propagation
        then runs one ordinary launch per round instead of a cooperative
        grid."""
        st = _lib().ibip_set_shared_device(self._h, int(bool(on)))
        if st != OK:
            raise IbipError("ibip_set_shared_device", st)

    def set_literal_cluster(self, cluster: int):
        """CTAs per image cluster of invade_literal_batched (0 = automatic)."""
        st = _lib().ibip_set_literal_cluster(self._h, int(cluster))
        if st != OK:
            raise IbipError("ibip_set_literal_cluster", st)

    def invade_literal_batched(self, images, inlets=0, max_steps=None):
        """The paper-literal invasion of many images, each on a thread-block
        cluster of its own, in one launch (ibip_invade_literal_batched).
        Returns (list of dicts with seq, cstep, step_r2, step_count, K,
        status; the cluster size used)."""
        n = len(images)
        inl = inlets if isinstance(inlets, (list, tuple)) else [inlets] * n
        jobs = (LiteralJob * n)()
        outs = []
        for j, im in enumerate(images):
            _need(im, torch.uint8, "image")
            dev, N = im.device, im.numel()
            r = {"seq": torch.empty(im.shape, dtype=torch.int32, device=dev),
                 "cstep": torch.empty(im.shape, dtype=torch.int32, device=dev),
                 "step_r2": torch.empty(max(N, 1), dtype=torch.int32, device=dev),
                 "step_count": torch.empty(max(N, 1), dtype=torch.int32, device=dev)}
            J = jobs[j]
            J.image = im.data_ptr()
            J.dims = _dims(im.shape)
            J.inlet = int(inl[j])
            J.dt2 = None
            J.max_steps = -1 if max_steps is None else int(max_steps)
            J.seq, J.cstep = r["seq"].data_ptr(), r["cstep"].data_ptr()
            J.step_r2, J.step_count = r["step_r2"].data_ptr(), r["step_count"].data_ptr()
            J.capacity_steps = N
            outs.append(r)
        cs = C.c_int(0)
        self._stream()
        st = _lib().ibip_invade_literal_batched(self._h, n, jobs, C.byref(cs))
        if st not in (OK, ERR_STEP_LIMIT):
            raise IbipError("ibip_invade_literal_batched", st)
        for r, J in zip(outs, jobs):
            K = int(J.n_steps)
            r["K"], r["status"] = K, int(J.status)
            r["step_r2"], r["step_count"] = r["step_r2"][:K], r["step_count"][:K]
        return outs, int(cs.value)

    def trapping(self, seq, outlet=1, rerank=False, seq_out=True):
        _need(seq, torch.int32, "seq")
        tr = torch.empty(seq.shape, dtype=torch.uint8, device=seq.device)
        so = torch.empty_like(seq) if seq_out else None
        self._stream()
        st = _lib().ibip_trapping(self._h, _ptr(seq), _dims(seq.shape), int(outlet), int(bool(rerank)), _ptr(tr),
                                  _ptr(so))
        if st != OK:
            raise IbipError("ibip_trapping", st)
        return tr, so

    def trapping_rerank(self, seq, step_r2, outlet=1):
        """Trapping with re-ranking and the surviving steps' radii
        (ibip_trapping_ex).  Returns (trapped, seq_out, step_r2_out)."""
        _need(seq, torch.int32, "seq")
        K = int(step_r2.numel())
        tr = torch.empty(seq.shape, dtype=torch.uint8, device=seq.device)
        so = torch.empty(seq.shape, dtype=torch.int32, device=seq.device)
        r2o = torch.empty(max(K, 1), dtype=torch.int32, device=seq.device)
        r2 = step_r2.contiguous()
        n = C.c_int64(0)
        self._stream()
        st = _lib().ibip_trapping_ex(self._h, _ptr(seq), _dims(seq.shape), int(outlet), _ptr(tr), _ptr(so), _ptr(r2),
                                     K, _ptr(r2o), C.byref(n))
        if st != OK:
            raise IbipError("ibip_trapping_ex", st)
        return tr, so, r2o[:int(n.value)]

    def size_image(self, seq, step_r2):
        """Squared radius of the sphere that invaded each voxel (ibip_size_image)."""
        _need(seq, torch.int32, "seq")
        out = torch.empty(seq.shape, dtype=torch.int32, device=seq.device)
        r2 = step_r2.contiguous()
        self._stream()
        st = _lib().ibip_size_image(self._h, _ptr(seq), _dims(seq.shape), _ptr(r2), int(r2.numel()), _ptr(out))
        if st != OK:
            raise IbipError("ibip_size_image", st)
        return out

    def morph_drainage(self, image, dt2, levels, inlet=0, dilate_levels=None):
        """Opening drainage: level i erodes at dt2 >= levels[i] and dilates by
        d^2 < dilate_levels[i] (default: the same bounds).  Returns (level,
        counts)."""
        _need(image, torch.uint8, "image")
        _need(dt2, torch.int32, "dt2")
        T = (C.c_int32 * max(len(levels), 1))(*[int(t) for t in levels])
        Td = None
        if dilate_levels is not None:
            if len(dilate_levels) != len(levels):
                raise ValueError("dilate_levels must have one bound per level")
            Td = (C.c_int32 * max(len(levels), 1))(*[int(t) for t in dilate_levels])
        cnt = (C.c_int64 * max(len(levels), 1))()
        lev = torch.empty(image.shape, dtype=torch.int32, device=image.device)
        self._stream()
        st = _lib().ibip_morph_drainage_ex(self._h, _ptr(image), _ptr(dt2), _dims(image.shape), int(inlet), T, Td,
                                           len(levels), _ptr(lev), cnt)
        if st != OK:
            raise IbipError("ibip_morph_drainage_ex", st)
        return lev, [int(c) for c in cnt[:len(levels)]]

    def invade_batched(self, images, inlets=0, outlets=1, trapping=True, curve=True, voxel_m=5e-6, sigma=0.072,
                       theta_deg=180.0, check=True):
        """EDT, invasion, trapping and Pc curve of many images in one call.
        `images`: list of 3-D CUDA uint8 tensors; `inlets` / `outlets`: a face
        or a list of faces.  Returns one dict per image with seq, step_r2,
        step_centre, K, status and (if requested) trapped, seq_out, S, Pc."""
        n = len(images)
        inl = inlets if isinstance(inlets, (list, tuple)) else [inlets] * n
        outl = outlets if isinstance(outlets, (list, tuple)) else [outlets] * n
        for im in images:
            _need(im, torch.uint8, "image")
        dev = images[0].device
        sizes = [im.numel() for im in images]
        offs, tot = [], 0
        for N in sizes:
            offs.append(tot)
            tot += max(N, 1)
        # one buffer per output kind, every image a slice of it
        pool = {"seq": torch.empty(tot, dtype=torch.int32, device=dev),
                "step_r2": torch.empty(tot, dtype=torch.int32, device=dev),
                "step_centre": torch.empty(tot, dtype=torch.int32, device=dev)}
        if trapping:
            pool["trapped"] = torch.empty(tot, dtype=torch.uint8, device=dev)
            pool["seq_out"] = torch.empty(tot, dtype=torch.int32, device=dev)
        if curve:
            pool["S"] = torch.empty(tot, dtype=torch.float32, device=dev)
            pool["Pc"] = torch.empty(tot, dtype=torch.float32, device=dev)
        base = {k: (v.data_ptr(), v.element_size()) for k, v in pool.items()}
        arr = (Job * n)()
        vm, sg, th = float(voxel_m), float(sigma), float(theta_deg)
        for j, im in enumerate(images):
            J, o = arr[j], offs[j]
            J.image = im.data_ptr()
            J.dims = _dims(im.shape)
            J.inlet, J.outlet = int(inl[j]), int(outl[j]) if trapping else -1
            J.dt2 = None
            J.seq = base["seq"][0] + 4 * o
            J.step_r2 = base["step_r2"][0] + 4 * o
            J.step_centre = base["step_centre"][0] + 4 * o
            J.capacity_steps = sizes[j]
            J.trapped = base["trapped"][0] + o if trapping else None
            J.seq_out = base["seq_out"][0] + 4 * o if trapping else None
            J.sat_per_step = base["S"][0] + 4 * o if curve else None
            J.pc_per_step = base["Pc"][0] + 4 * o if curve else None
            J.voxel_m, J.sigma, J.theta_deg = vm, sg, th
        self._stream()
        st = _lib().ibip_invade_batched(self._h, n, arr)
        if check and st != OK:
            raise IbipError("ibip_invade_batched", st)
        res = []
        for j, im in enumerate(images):
            o, N, K = offs[j], sizes[j], int(arr[j].n_steps)
            r = {"K": K, "status": int(arr[j].status)}
            for key, v in pool.items():
                if key in ("seq", "trapped", "seq_out"):
                    r[key] = v[o:o + N].view(im.shape)
                else:
                    r[key] = v[o:o + min(K, N)]
            res.append(r)
        return res

    def equal_saturation(self, seq, level, n_steps, n_levels):
        """Equal-saturation comparison with opening levels (Section 3.1.1):
        returns (k, diff, n) as lists, one entry per level."""
        _need(seq, torch.int32, "seq")
        _need(level, torch.int32, "level")
        L = int(n_levels)
        k, d, n = (C.c_int64 * L)(), (C.c_int64 * L)(), (C.c_int64 * L)()
        self._stream()
        st = _lib().ibip_equal_saturation(self._h, _ptr(seq), _ptr(level), _dims(seq.shape), int(n_steps), L,
                                          k, d, n)
        if st != OK:
            raise IbipError("ibip_equal_saturation", st)
        return list(k), list(d), list(n)

    def pc_envelope(self, seq, step_r2, levels):
        """Drainage envelope at opening levels (ibip_pc_envelope): per level,
        (steps taken before the running-minimum sphere drops below it,
        voxels invaded by then)."""
        _need(seq, torch.int32, "seq")
        K = int(step_r2.numel())
        L = len(levels)
        T = (C.c_int32 * max(L, 1))(*[int(t) for t in levels])
        ks = (C.c_int64 * max(L, 1))()
        ns = (C.c_int64 * max(L, 1))()
        self._stream()
        st = _lib().ibip_pc_envelope(self._h, _ptr(seq), _dims(seq.shape), _ptr(step_r2) if K else None, K, T, L,
                                     ks, ns)
        if st != OK:
            raise IbipError("ibip_pc_envelope", st)
        return [int(x) for x in ks[:L]], [int(x) for x in ns[:L]]

    def pc_curve(self, seq, step_r2, voxel_m=5e-6, sigma=0.072, theta_deg=180.0, sat_image=False):
        _need(seq, torch.int32, "seq")
        K = int(step_r2.numel())
        dev = seq.device
        S = torch.empty(max(K, 1), dtype=torch.float32, device=dev)
        P = torch.empty(max(K, 1), dtype=torch.float32, device=dev)
        img = torch.empty(seq.shape, dtype=torch.float32, device=dev) if sat_image else None
        r2 = step_r2.contiguous()
        self._stream()
        st = _lib().ibip_pc_curve(self._h, _ptr(seq), _dims(seq.shape), _ptr(r2), K, float(voxel_m), float(sigma),
                                  float(theta_deg), _ptr(S), _ptr(P), _ptr(img))
        if st != OK:
            raise IbipError("ibip_pc_curve", st)
        return S[:K], P[:K], img


class Server:
    """Continuous-batching request loop (ibip_server_*): jobs are admitted in
    arrival order as slots and arena memory free up, and run concurrently on
    the slots' streams.  `mem_budget` bytes of device memory are allocated
    up front."""

    def __init__(self, ctx: Context, mem_budget: int, max_slots: int = 16):
        h = C.c_void_p()
        st = _lib().ibip_server_create(C.byref(h), ctx._h, int(mem_budget), int(max_slots))
        if st != OK:
            raise IbipError("ibip_server_create", st)
        self._h = h
        self.device = ctx.device
        self._live = {}   # ticket -> (job, image, outputs): kept alive until collected

    def submit(self, image, inlet=0, outlet=1, trapping=True, curve=True, voxel_m=5e-6, sigma=0.072,
               theta_deg=180.0) -> int:
        """Queues the whole path for one image; returns its ticket.  The
        image and the outputs are read and written on a slot's stream, so
        the current stream is synchronised first (the image must be ready)."""
        J = Job()
        r = _fill_job(J, image, int(inlet), int(outlet), trapping, curve, voxel_m, sigma, theta_deg)
        torch.cuda.current_stream(image.device).synchronize()
        t = C.c_uint64()
        st = _lib().ibip_server_submit(self._h, C.byref(J), C.byref(t))
        if st != OK:
            raise IbipError("ibip_server_submit", st)
        self._live[t.value] = (J, image, r)
        return t.value

    def _collect(self, ticket, done, res):
        if not done.value:
            return None
        _, _, r = self._live.pop(ticket)
        K = int(res.n_steps)
        r.update(K=K, status=int(res.status), slot=int(res.slot), t_submit_ns=int(res.t_submit_ns),
                 t_start_ns=int(res.t_start_ns), t_end_ns=int(res.t_end_ns), mem_reserved=int(res.mem_reserved),
                 mem_used=int(res.mem_used))
        return _trim(r, K)

    def poll(self, ticket):
        """The job's result dict if it has completed (collected once), else None."""
        done, res = C.c_int(), Result()
        st = _lib().ibip_server_poll(self._h, int(ticket), C.byref(done), C.byref(res))
        if st != OK:
            raise IbipError("ibip_server_poll", st)
        return self._collect(ticket, done, res)

    def wait(self, ticket, timeout=None):
        """Blocks until the job completes (or `timeout` seconds pass: None)."""
        done, res = C.c_int(), Result()
        us = -1 if timeout is None else int(timeout * 1e6)
        st = _lib().ibip_server_wait(self._h, int(ticket), us, C.byref(done), C.byref(res))
        if st != OK:
            raise IbipError("ibip_server_wait", st)
        return self._collect(ticket, done, res)

    def stats(self) -> dict:
        v = (C.c_int64 * 9)()
        _lib().ibip_server_stats(self._h, v, 9)
        keys = ("submitted", "completed", "running", "waiting", "arena_used", "arena_bytes", "peak_running",
                "peak_arena_used", "launches")
        return dict(zip(keys, (int(x) for x in v)))

    def close(self):
        if getattr(self, "_h", None):
            _lib().ibip_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def route_pick(loads, capacities, footprint) -> int:
    """The routing rule of ibip_route_pick (host only): the replica with the
    least outstanding work among those whose arena holds `footprint` bytes,
    the lowest index on ties; -1 when none can hold it."""
    n = len(loads)
    if n < 1 or len(capacities) != n:
        raise ValueError("one capacity per load, at least one replica")
    L = (C.c_int64 * n)(*[int(x) for x in loads])
    Cp = (C.c_int64 * n)(*[int(x) for x in capacities])
    r = _lib().ibip_route_pick(n, L, Cp, int(footprint))
    if r == ERR_OOM:
        return -1
    if r < 0:
        raise IbipError("ibip_route_pick", r)
    return r


def route_requests(voxels, n_replicas, capacity=None, footprints=None):
    """Static routing of a request stream over `n_replicas` processes (one
    GPU each) that cannot see each other's progress: request j goes, in
    arrival order, by ibip_route_pick to the replica with the fewest voxels
    routed so far (among those whose arena `capacity` holds its footprint,
    when given).  Every process computes the same assignment from the same
    stream, so no message is needed.  Returns the replica of each request."""
    loads = [0] * n_replicas
    caps = [capacity if capacity is not None else (1 << 62)] * n_replicas
    out = []
    for j, v in enumerate(voxels):
        r = route_pick(loads, caps, 0 if footprints is None else footprints[j])
        if r < 0:
            raise ValueError("request %d fits no replica" % j)
        loads[r] += int(v)
        out.append(r)
    return out


class Router:
    """Serving replicas: one continuous-batching server per entry of
    `devices` (a device may appear more than once).  Each request goes to
    the replica with the least outstanding work (ibip_router_route); its
    image is copied to that replica's device and its outputs are allocated
    there."""

    def __init__(self, devices, mem_budget: int, max_slots: int = 16):
        devs = [int(torch.device(d).index if not isinstance(d, int) else d) for d in devices]
        arr = (C.c_int * len(devs))(*devs)
        h = C.c_void_p()
        st = _lib().ibip_router_create(C.byref(h), len(devs), arr, int(mem_budget), int(max_slots))
        if st != OK:
            raise IbipError("ibip_router_create", st)
        self._h = h
        self.devices = devs
        self._live = {}

    def route(self, shape):
        """(replica, device index) a job of this shape would go to now."""
        r, d = C.c_int(), C.c_int()
        st = _lib().ibip_router_route(self._h, _dims(shape), 1, C.byref(r), C.byref(d))
        if st != OK:
            raise IbipError("ibip_router_route", st)
        return r.value, d.value

    def submit(self, image, inlet=0, outlet=1, trapping=True, curve=True, voxel_m=5e-6, sigma=0.072,
               theta_deg=180.0) -> int:
        """Routes one request: the image (a uint8 tensor on the host or any
        device) goes to the chosen replica's device; returns a ticket."""
        replica, dev = self.route(image.shape)
        im = image.to(torch.device("cuda", dev), non_blocking=False).contiguous()
        J = Job()
        r = _fill_job(J, im, int(inlet), int(outlet), trapping, curve, voxel_m, sigma, theta_deg)
        torch.cuda.current_stream(im.device).synchronize()
        t = C.c_uint64()
        st = _lib().ibip_router_submit(self._h, replica, C.byref(J), C.byref(t))
        if st != OK:
            raise IbipError("ibip_router_submit", st)
        self._live[t.value] = (J, im, r)
        return t.value

    def wait(self, ticket, timeout=None):
        """The job's result dict (with its `replica`) once complete, else None
        after `timeout` seconds."""
        done, res, rep = C.c_int(), Result(), C.c_int()
        us = -1 if timeout is None else int(timeout * 1e6)
        st = _lib().ibip_router_wait(self._h, int(ticket), us, C.byref(done), C.byref(res), C.byref(rep))
        if st != OK:
            raise IbipError("ibip_router_wait", st)
        if not done.value:
            return None
        _, _, r = self._live.pop(ticket)
        K = int(res.n_steps)
        r.update(K=K, status=int(res.status), slot=int(res.slot), replica=int(rep.value),
                 t_submit_ns=int(res.t_submit_ns), t_start_ns=int(res.t_start_ns), t_end_ns=int(res.t_end_ns))
        return _trim(r, K)

    def stats(self, replica) -> dict:
        v = (C.c_int64 * 12)()
        st = _lib().ibip_router_stats(self._h, int(replica), v, 12)
        if st != OK:
            raise IbipError("ibip_router_stats", st)
        keys = ("device", "routed", "outstanding_voxels", "submitted", "completed", "running", "waiting",
                "arena_used", "arena_bytes", "peak_running", "peak_arena_used", "launches")
        return dict(zip(keys, (int(x) for x in v)))

    def close(self):
        if getattr(self, "_h", None):
            _lib().ibip_router_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default = {}


def context(device=None) -> Context:
    """A cached context per device."""
    idx = torch.cuda.current_device() if device is None else int(device)
    c = _default.get(idx)
    if c is None:
        c = _default[idx] = Context(idx)
    return c
