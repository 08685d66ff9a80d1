"""Plain FP64 CPU oracle for the parallel-in-time Newton ODE solver (arXiv 2511.01465).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use this package; the product library never imports it.  The
arithmetic lives in ``pitn_oracle.c`` (plain C, one core, FP64, compiled with
``-ffp-contract=off``); this module only builds that file with gcc and
marshals numpy arrays through ctypes.  See the C file's header for which
equation each routine follows.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pitn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None
_variant_libs = {}

# Rounding variants of the same C file (test builds only): each computes the
# same mathematics in another rounding order.  They measure how far rounding
# alone moves results whose decisions compare rounded values (the guard's cut
# index and with it the Newton count of a guarded solve).
_FMA = ["-ffp-contract=fast"] + (["-mfma"] if platform.machine() in ("x86_64", "AMD64") else [])
VARIANTS = {
    "fma": _FMA,                                        # every a*b + c contracted
    "rev": ["-DORACLE_SUM_REVERSED"],                   # matrix-vector sums last index first
    "diff": ["-DORACLE_RESID_DIFF_FIRST"],              # residual (x_n - x_{n-1}) - h f
    "blk4": ["-DORACLE_BLOCK=4"],                       # recursion bracketed in blocks of 4
    "blk64": ["-DORACLE_BLOCK=64"],                     # ... of 64
    "fma_rev_diff_blk64": _FMA + ["-DORACLE_SUM_REVERSED", "-DORACLE_RESID_DIFF_FIRST",
                                  "-DORACLE_BLOCK=64"],
}
# A reduced-precision variant (test builds only): the recursion of eq. 3.13
# carried in a 48-bit significand, the precision of a scan in pairs of 24-bit
# floats; kept apart from VARIANTS, which are FP64 rounding orders only.
SCAN_VARIANTS = {
    "s48": ["-DORACLE_SCAN_BITS=48"],
}

# identifiers understood by the C oracle
LORENZ63, VDP, LINEAR_OSC, FKPP, LOGISTIC, DAHLQUIST, ROBERTSON = 1, 2, 3, 4, 5, 6, 7
EULER, RK4, BACKWARD_EULER, TRAPEZOID = 0, 1, 2, 3
OK, NOT_CONVERGED, NONFINITE = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False, variant: str | None = None) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no FP
    contraction), or one of its rounding VARIANTS (or SCAN_VARIANTS) into
    liboracle_<variant>.so."""
    lib_path = _LIB if variant is None else os.path.join(_BUILD, f"liboracle_{variant}.so")
    vflags = [] if variant is None else {**VARIANTS, **SCAN_VARIANTS}[variant]
    flags = (["-ffp-contract=off"] if "-ffp-contract=fast" not in vflags else []) + vflags
    with _lock:
        if (not force and os.path.exists(lib_path)
                and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC)):
            return lib_path
        os.makedirs(_BUILD, exist_ok=True)
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11"] + flags + ["-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib_path)
        return lib_path


def _load(variant: str | None = None):
    global _lib
    if variant is not None:
        if variant not in _variant_libs:
            _variant_libs[variant] = _declare(ctypes.CDLL(build(variant=variant)))
        return _variant_libs[variant]
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(lib):
    """Argument types of the oracle's C entry points."""
    c_int, c_i64, c_d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.oracle_nparams.argtypes = [c_int]
    lib.oracle_rhs.argtypes = [c_int, _dp, c_int, _dp, _dp]
    lib.oracle_rhs_jac.argtypes = [c_int, _dp, c_int, _dp, _dp]
    lib.oracle_rhs_dparam.argtypes = [c_int, _dp, c_int, _dp, _dp]
    lib.oracle_step.argtypes = [c_int, c_int, _dp, c_int, c_d, _dp, _dp, _dp, _dp]
    lib.oracle_sequential.argtypes = [c_int, c_int, _dp, _dp, c_d, c_i64, c_int, _dp]
    lib.oracle_residual.argtypes = [c_int, c_int, _dp, _dp, c_d, c_i64, c_int, _dp, _dp, _dp,
                                    ctypes.POINTER(c_int)]
    lib.oracle_combine.argtypes = [c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.oracle_affine_scan.argtypes = [c_i64, c_int, _dp, _dp, _dp]
    lib.oracle_newton.argtypes = [c_int, c_int, _dp, _dp, c_d, c_i64, c_int, c_d, c_int, c_d,
                                  _dp, _dp, _dp, _i32p, _i32p, _i64p, _i64p]
    lib.oracle_newton_batch.argtypes = [c_int, c_int, c_i64, _dp, _dp, _dp, _i64p, c_int, c_d,
                                        c_int, c_d, _dp, _i64p, _i32p, _i32p, _dp]
    lib.oracle_adjoint.argtypes = [c_int, c_int, _dp, _dp, c_d, c_i64, c_int, _dp, _dp, _dp,
                                   _dp, _dp]
    return lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _need(a, size, what):
    """The C routines read exactly `size` doubles from each buffer: refuse others."""
    if a.size != size:
        raise ValueError(f"{what}: expected {size} values, got {a.size}")
    return a


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle call failed with code {rc}")


def nparams(sys: int) -> int:
    return _load().oracle_nparams(sys)


def rhs(sys, p, x):
    p, x = _f64(p), _f64(x)
    _need(p, nparams(sys), "p")
    out = np.empty_like(x)
    _check(_load().oracle_rhs(sys, _ptr(p), x.size, _ptr(x), _ptr(out)))
    return out


def rhs_jac(sys, p, x):
    p, x = _f64(p), _f64(x)
    _need(p, nparams(sys), "p")
    d = x.size
    out = np.empty((d, d))
    _check(_load().oracle_rhs_jac(sys, _ptr(p), d, _ptr(x), _ptr(out)))
    return out


def rhs_dparam(sys, p, x):
    p, x = _f64(p), _f64(x)
    _need(p, nparams(sys), "p")
    d = x.size
    out = np.empty((d, nparams(sys)))
    _check(_load().oracle_rhs_dparam(sys, _ptr(p), d, _ptr(x), _ptr(out)))
    return out


def step(sys, p, h, x, method=EULER, jac=False, dparam=False):
    """phi(x) and optionally dphi/dx, dphi/dp."""
    p, x = _f64(p), _f64(x)
    _need(p, nparams(sys), "p")
    d = x.size
    phi = np.empty(d)
    J = np.empty((d, d)) if jac else None
    G = np.empty((d, nparams(sys))) if dparam else None
    _check(_load().oracle_step(sys, method, _ptr(p), d, float(h), _ptr(x), _ptr(phi), _ptr(J), _ptr(G)))
    return phi, J, G


def sequential(sys, p, x0, h, N, method=EULER):
    p, x0 = _f64(p), _f64(x0)
    _need(p, nparams(sys), "p")
    d = x0.size
    traj = np.empty((int(N), d))
    _check(_load().oracle_sequential(sys, method, _ptr(p), _ptr(x0), float(h), int(N), d, _ptr(traj)))
    return traj


def residual(sys, p, x0, h, traj, method=EULER):
    """(r [N][d], ||r||_inf, nonfinite flag) of eq. (3.8) for trajectory x_1..x_N."""
    p, x0, traj = _f64(p), _f64(x0), _f64(traj)
    N, d = traj.shape
    _need(p, nparams(sys), "p"), _need(x0, d, "x0")
    r = np.empty_like(traj)
    res = ctypes.c_double()
    nf = ctypes.c_int()
    _check(_load().oracle_residual(sys, method, _ptr(p), _ptr(x0), float(h), N, d, _ptr(traj),
                                   _ptr(r), ctypes.byref(res), ctypes.byref(nf)))
    return r, res.value, bool(nf.value)


def combine(A2, b2, A1, b1):
    """(A2, b2) (x) (A1, b1) of eq. (3.3)."""
    A2, b2, A1, b1 = map(_f64, (A2, b2, A1, b1))
    d = b1.size
    _need(A2, d * d, "A2"), _need(A1, d * d, "A1"), _need(b2, d, "b2")
    A, b = np.empty((d, d)), np.empty(d)
    _check(_load().oracle_combine(d, _ptr(A2), _ptr(b2), _ptr(A1), _ptr(b1), _ptr(A), _ptr(b)))
    return A, b


def affine_scan(A, c):
    """Sequential states z[n] of z <- A_n z + c_n from z = 0 (element 0's matrix ignored)."""
    A, c = _f64(A), _f64(c)
    N, d = c.shape
    _need(A, N * d * d, "A")
    z = np.empty_like(c)
    _check(_load().oracle_affine_scan(N, d, _ptr(A), _ptr(c), _ptr(z)))
    return z


def newton(sys, p, x0, h, N, tol, max_iter, guard_B=0.0, guess=None, method=EULER, variant=None):
    """Returns dict(traj, res_hist, iters, status, guard_index, cuts).

    cuts[k] is the guard cut q of Newton step k (N when nothing was cut).
    variant: None for the oracle itself, or a key of VARIANTS (a rounding
    variant, test use only)."""
    p, x0 = _f64(p), _f64(x0)
    _need(p, nparams(sys), "p")
    d = x0.size
    traj = np.empty((int(N), d))
    hist = np.full(max_iter + 1, np.nan)
    cuts = np.full(max_iter + 1, -1, dtype=np.int64)
    iters, status, gi = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    g = None
    if guess is not None:   # a scalar or d-vector fills every step; else one row per step
        g = _f64(np.broadcast_to(_f64(guess), (int(N), d)))
    _check(_load(variant).oracle_newton(sys, method, _ptr(p), _ptr(x0), float(h), int(N), d, float(tol),
                                        int(max_iter), float(guard_B), _ptr(g), _ptr(traj), _ptr(hist),
                                        ctypes.byref(iters), ctypes.byref(status), ctypes.byref(gi),
                                        cuts.ctypes.data_as(_i64p)))
    return dict(traj=traj, res_hist=hist[: iters.value + 1], iters=iters.value,
                status=status.value, guard_index=gi.value, cuts=cuts[cuts >= 0])


def newton_batch(sys, params, x0, h, N, tol, max_iter, guard_B=0.0, method=EULER):
    params, x0, h = _f64(params), _f64(x0), _f64(h)
    N = np.ascontiguousarray(np.asarray(N, dtype=np.int64))
    B, d = x0.shape
    _need(params, B * nparams(sys), "params"), _need(h, B, "h"), _need(N, B, "N")
    traj = np.empty((int(N.sum()), d))
    offsets = np.empty(B + 1, dtype=np.int64)
    iters = np.empty(B, dtype=np.int32)
    status = np.empty(B, dtype=np.int32)
    res = np.empty(B)
    _check(_load().oracle_newton_batch(
        sys, method, B, _ptr(params), _ptr(x0), _ptr(h), N.ctypes.data_as(_i64p), d, float(tol),
        int(max_iter), float(guard_B), _ptr(traj), offsets.ctypes.data_as(_i64p),
        iters.ctypes.data_as(_i32p), status.ctypes.data_as(_i32p), _ptr(res)))
    return dict(traj=traj, offsets=offsets, iters=iters, status=status, res=res)


def adjoint(sys, p, x0, h, traj, grad_traj=None, grad_xN=None, method=EULER):
    """(dL/dx0, dL/dp) by the reverse recursion."""
    p, x0, traj = _f64(p), _f64(x0), _f64(traj)
    N, d = traj.shape
    _need(p, nparams(sys), "p"), _need(x0, d, "x0")
    gt = _need(_f64(grad_traj), N * d, "grad_traj") if grad_traj is not None else None
    gN = _need(_f64(grad_xN), d, "grad_xN") if grad_xN is not None else None
    gx0 = np.empty(d)
    gp = np.empty(nparams(sys))
    _check(_load().oracle_adjoint(sys, method, _ptr(p), _ptr(x0), float(h), N, d, _ptr(traj),
                                  _ptr(gt), _ptr(gN), _ptr(gx0), _ptr(gp)))
    return gx0, gp
