"""ctypes binding of ``libpitn.so`` (the C ABI of ``include/pitn.h``).

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must be
float64 (int64 for lengths/offsets, int32 for counts/statuses) and
contiguous.  Their raw pointers are passed through; the library detects
host vs device memory itself.  If the library is missing this module raises
on first use: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpitn.so")

# return codes
PITN_OK, PITN_NOT_CONVERGED, PITN_NONFINITE = 0, 1, 2
PITN_EINVAL, PITN_ENOMEM, PITN_ECUDA, PITN_ETIMEOUT, PITN_EUNSUPPORTED = -1, -2, -3, -4, -5
# systems
PITN_LORENZ63, PITN_VDP, PITN_LINEAR_OSC, PITN_FKPP, PITN_LOGISTIC = 1, 2, 3, 4, 5
PITN_DAHLQUIST, PITN_ROBERTSON = 6, 7
# one-step maps
PITN_STEP_EULER, PITN_STEP_RK4, PITN_STEP_BACKWARD_EULER, PITN_STEP_TRAPEZOID = 0, 1, 2, 3
# failure injection (pitn_debug_inject)
PITN_DEBUG_RESET, PITN_DEBUG_FAIL_ALLOCS, PITN_DEBUG_GRID_WAIT_NS = 0, 1, 2
PITN_DEBUG_LOAD_POLLS, PITN_DEBUG_MMA_POLLS = 3, 4
# precisions
PITN_PREC_FP64, PITN_PREC_MIXED_BF16, PITN_PREC_MIXED_FP32, PITN_PREC_FP64_FF, PITN_PREC_MIXED_TF32 = 0, 1, 2, 3, 4


class pitn_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("final_res", ctypes.c_double), ("guard_index", ctypes.c_int64)]


class pitn_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tile_elems", ctypes.c_int32),
                ("guard_B", ctypes.c_double), ("guess", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("res_history", ctypes.c_void_p),
                ("method", ctypes.c_int32), ("cut_history", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Loads libpitn.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                               "`python -m paper_2511_01465_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, d, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
        L.pitn_solve.argtypes = [c_int, vp, vp, d, i64, c_int, d, c_int, vp]
        L.pitn_solve.restype = c_int
        L.pitn_solve_ex.argtypes = [c_int, vp, vp, d, i64, c_int, d, c_int, vp,
                                    ctypes.POINTER(pitn_options), ctypes.POINTER(pitn_result)]
        L.pitn_solve_ex.restype = c_int
        L.pitn_solve_batch.argtypes = [c_int, i64, vp, vp, vp, vp, c_int, d, c_int, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(pitn_options)]
        L.pitn_solve_batch.restype = c_int
        L.pitn_backward.argtypes = [c_int, i64, vp, vp, vp, vp, c_int, vp, vp, vp, c_int, vp, vp,
                                    ctypes.POINTER(pitn_options)]
        L.pitn_backward.restype = c_int
        L.pitn_num_params.argtypes = [c_int]
        L.pitn_num_params.restype = c_int
        L.pitn_status_string.argtypes = [c_int]
        L.pitn_status_string.restype = ctypes.c_char_p
        L.pitn_release_workspace.argtypes = []
        L.pitn_release_workspace.restype = c_int
        L.pitn_launch_count.argtypes = []
        L.pitn_launch_count.restype = i64
        L.pitn_batch_work.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.pitn_batch_work.restype = c_int
        L.pitn_probe_fma_rate.argtypes = [c_int, ctypes.POINTER(d)]
        L.pitn_probe_fma_rate.restype = c_int
        L.pitn_debug_inject.argtypes = [c_int, i64]
        L.pitn_debug_inject.restype = c_int
        L.pitn_shard_create.argtypes = [c_int, vp, d, i64, c_int, d, vp, ctypes.POINTER(vp)]
        L.pitn_shard_create.restype = c_int
        L.pitn_shard_pass.argtypes = [vp, vp, c_int, vp, i64, vp, vp]
        L.pitn_shard_pass.restype = c_int
        L.pitn_shard_carry.argtypes = [vp, i64, vp, vp]
        L.pitn_shard_carry.restype = c_int
        L.pitn_shard_update.argtypes = [vp, vp, vp, vp]
        L.pitn_shard_update.restype = c_int
        L.pitn_shard_finalize.argtypes = [vp, vp, vp, i64, vp]
        L.pitn_shard_finalize.restype = c_int
        L.pitn_shard_destroy.argtypes = [vp]
        L.pitn_shard_destroy.restype = c_int
        L.pitn_solve_noalloc.argtypes = [c_int, vp, vp, d, i64, c_int, d, c_int, d, vp,
                                          ctypes.POINTER(pitn_result)]
        L.pitn_solve_noalloc.restype = c_int
        L.pitn_affine_combine_delta.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        L.pitn_affine_combine_delta.restype = c_int
        L.pitn_affine_combine_delta_tf32.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        L.pitn_affine_combine_delta_tf32.restype = c_int
        L.pitn_tune_enable.argtypes = [c_int]
        L.pitn_tune_enable.restype = c_int
        L.pitn_tune_clear.argtypes = []
        L.pitn_tune_clear.restype = c_int
        L.pitn_tune_get.argtypes = [ctypes.c_char_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        L.pitn_tune_get.restype = c_int
        L.pitn_tune_set.argtypes = [ctypes.c_char_p, c_int, c_int]
        L.pitn_tune_set.restype = c_int
        L.pitn_timing_enable.argtypes = [c_int]
        L.pitn_timing_enable.restype = c_int
        L.pitn_timing_reset.argtypes = []
        L.pitn_timing_reset.restype = c_int
        L.pitn_timing_get.argtypes = [ctypes.c_char_p, ctypes.POINTER(d), ctypes.POINTER(i64)]
        L.pitn_timing_get.restype = c_int
        _lib = L
        return L


def _ptr(a, dtype=np.float64):
    """Raw data pointer of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch.Tensor
        import torch
        want = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def make_options(precision=PITN_PREC_FP64, tile_elems=0, guard_B=0.0, guess=None, stream=None,
                 res_history=None, method=PITN_STEP_EULER, cut_history=None):
    o = pitn_options()
    o.method = int(method)
    o.precision = int(precision)
    o.tile_elems = int(tile_elems)
    o.guard_B = float(guard_B)
    o.guess = _ptr(guess)
    o.stream = ctypes.c_void_p(int(stream)) if stream is not None else None
    o.res_history = _ptr(res_history)
    o.cut_history = _ptr(cut_history, np.int64)
    o._keep = (guess, res_history, cut_history)
    return o


def _stream_handle(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def pitn_solve(system_id, params, x0, h, N, d, tol, max_iter, traj_out):
    return lib().pitn_solve(int(system_id), _ptr(params), _ptr(x0), float(h), int(N), int(d),
                            float(tol), int(max_iter), _ptr(traj_out))


def pitn_solve_ex(system_id, params, x0, h, N, d, tol, max_iter, traj_out, opt=None):
    """Returns (code, pitn_result)."""
    res = pitn_result()
    optp = ctypes.byref(opt) if opt is not None else None
    rc = lib().pitn_solve_ex(int(system_id), _ptr(params), _ptr(x0), float(h), int(N), int(d),
                             float(tol), int(max_iter), _ptr(traj_out), optp, ctypes.byref(res))
    return rc, res


def pitn_solve_batch(system_id, B, params, x0, h, N, d, tol, max_iter, traj_out, offsets_out,
                     iters_out, status_out, res_out=None, opt=None):
    optp = ctypes.byref(opt) if opt is not None else None
    return lib().pitn_solve_batch(int(system_id), int(B), _ptr(params), _ptr(x0), _ptr(h),
                                  _ptr(N, np.int64), int(d), float(tol), int(max_iter),
                                  _ptr(traj_out), _ptr(offsets_out, np.int64),
                                  _ptr(iters_out, np.int32), _ptr(status_out, np.int32),
                                  _ptr(res_out), optp)


def pitn_backward(system_id, B, params, x0, h, N, d, traj, grad_traj, grad_xN, ckpt_every,
                  grad_x0_out, grad_params_out, opt=None):
    optp = ctypes.byref(opt) if opt is not None else None
    return lib().pitn_backward(int(system_id), int(B), _ptr(params), _ptr(x0), _ptr(h),
                               _ptr(N, np.int64), int(d), _ptr(traj), _ptr(grad_traj),
                               _ptr(grad_xN), int(ckpt_every), _ptr(grad_x0_out),
                               _ptr(grad_params_out), optp)


def pitn_solve_noalloc(system_id, params, x0, h, N, d, tol, max_iter, guard_B, traj_out):
    """Allocation-free solve (small-state systems; traj_out must be device memory).
    Returns (code, pitn_result)."""
    res = pitn_result()
    rc = lib().pitn_solve_noalloc(int(system_id), _ptr(params), _ptr(x0), float(h), int(N), int(d),
                                  float(tol), int(max_iter), float(guard_B), _ptr(traj_out),
                                  ctypes.byref(res))
    return rc, res


def pitn_affine_combine_delta_tf32(n, S2, b2, S1, b1, S, b, stream=None):
    """pitn_affine_combine_delta with TF32 operands."""
    return pitn_affine_combine_delta(n, S2, b2, S1, b1, S, b, stream, _fn="pitn_affine_combine_delta_tf32")


def pitn_affine_combine_delta(n, S2, b2, S1, b1, S, b, stream=None, _fn="pitn_affine_combine_delta"):
    """n dense delta-form combines (float32 CUDA tensors, matrices [n][128][128] column-major)."""
    import torch
    def fp(t):
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError("float32 contiguous tensors expected")
        return ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(int(stream)) if stream is not None else None
    return getattr(lib(), _fn)(int(n), fp(S2), fp(b2), fp(S1), fp(b1), fp(S), fp(b), st)


def pitn_num_params(system_id):
    return lib().pitn_num_params(int(system_id))


def pitn_status_string(code):
    return lib().pitn_status_string(int(code)).decode()


def pitn_release_workspace():
    return lib().pitn_release_workspace()


def pitn_launch_count():
    return lib().pitn_launch_count()


def pitn_batch_work():
    """(steps evaluated, steps replayed) of the most recent batch solve."""
    ev, rep = ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().pitn_batch_work(ctypes.byref(ev), ctypes.byref(rep)), "pitn_batch_work")
    return int(ev.value), int(rep.value)


def pitn_tune_enable(on=True):
    return lib().pitn_tune_enable(1 if on else 0)


def pitn_tune_clear():
    return lib().pitn_tune_clear()


def pitn_tune_set(key, a, b):
    return lib().pitn_tune_set(key.encode(), int(a), int(b))


def pitn_tune_get(key):
    """(a, b) of a cached launch shape, or None."""
    a, b = ctypes.c_int(), ctypes.c_int()
    rc = lib().pitn_tune_get(key.encode(), ctypes.byref(a), ctypes.byref(b))
    return (a.value, b.value) if rc == 0 else None


def pitn_timing_enable(on=True):
    return lib().pitn_timing_enable(1 if on else 0)


def pitn_timing_reset():
    return lib().pitn_timing_reset()


def pitn_timing_get(kernel):
    """(total device ms, launches) of one kernel family since the last reset."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    rc = lib().pitn_timing_get(kernel.encode(), ctypes.byref(ms), ctypes.byref(n))
    if rc != 0:
        raise ValueError(rc)
    return ms.value, n.value


class PitnError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"{what}: {pitn_status_string(code)} ({code})")
        self.code = code


def check(code, what="pitn"):
    """Raises PitnError for negative (error) codes; returns the code otherwise."""
    if code < 0:
        raise PitnError(code, what)
    return code


def pitn_probe_fma_rate(kind):
    """Measured FMA rate of the current device (kind 0: FP64, 1: FP32), in
    thread FMAs per second."""
    v = ctypes.c_double()
    check(lib().pitn_probe_fma_rate(int(kind), ctypes.byref(v)), "pitn_probe_fma_rate")
    return v.value


def pitn_debug_inject(what, value=0):
    """Failure injection for tests of the error paths (see include/pitn.h)."""
    return lib().pitn_debug_inject(int(what), int(value))


def shard_create(system, params, h, n, d, guard_B=0.0, stream=None):
    """A time-shard plan (see include/pitn.h); params on the device or host."""
    plan = ctypes.c_void_p()
    st = ctypes.c_void_p(int(stream)) if stream is not None else None
    check(lib().pitn_shard_create(int(system), _ptr(params), float(h), int(n), int(d), float(guard_B), st,
                                  ctypes.byref(plan)), "pitn_shard_create")
    return plan
