"""Torch-facing helpers over the C ABI.

They allocate outputs as torch tensors, pass raw pointers to ``libpitn.so``
and turn its return codes into results; no arithmetic of the solver happens
here.
"""
from __future__ import annotations

import numpy as np

from . import pitn as P


def _torch():
    import torch
    return torch


def _as_f64(a, device):
    torch = _torch()
    t = torch.as_tensor(a, dtype=torch.float64)
    return t.to(device).contiguous()


def _stream_ptr(stream, device):
    torch = _torch()
    if stream is None:
        if str(device).startswith("cuda"):
            return torch.cuda.current_stream(device).cuda_stream
        return None
    return getattr(stream, "cuda_stream", stream)


def solve(system, params, x0, h, N, tol, max_iter, *, guard_B=0.0, precision=P.PITN_PREC_FP64,
          guess=None, device="cuda", stream=None, tile_elems=0, history=False, out=None,
          method=P.PITN_STEP_EULER):
    """Solves one IVP; returns (trajectory [N][d] tensor, info dict).

    info: iters (Newton updates), status (PITN_OK / NOT_CONVERGED / NONFINITE),
    final_res, guard_index and, with history=True, res_history (||h||_inf per
    residual evaluation) and cut_history (the guard cut of every computed
    Newton step).  Raises PitnError on a negative return code.
    """
    torch = _torch()
    x0_t = _as_f64(x0, device)
    p_t = _as_f64(params, device)
    d = int(x0_t.numel())
    traj = out if out is not None else torch.empty((int(N), d), dtype=torch.float64, device=device)
    g = _as_f64(guess, device) if guess is not None else None
    hist = np.full(max_iter + 1, np.nan) if history else None
    cuts = np.full(max_iter + 1, -1, dtype=np.int64) if history else None
    opt = P.make_options(precision=precision, tile_elems=tile_elems, guard_B=guard_B, guess=g,
                         stream=_stream_ptr(stream, device), res_history=hist, method=method,
                         cut_history=cuts)
    rc, res = P.pitn_solve_ex(system, p_t, x0_t, h, N, d, tol, max_iter, traj, opt)
    P.check(rc, "pitn_solve_ex")
    info = dict(iters=res.iters, status=res.status, final_res=res.final_res,
                guard_index=res.guard_index, code=rc)
    if history:
        info["res_history"] = hist[: res.iters + 1].copy()
        info["cut_history"] = cuts[cuts >= 0].copy()
    return traj, info


def solve_batch(system, params, x0, h, N, tol, max_iter, *, guard_B=0.0, device="cuda", stream=None,
                tile_elems=0, precision=0):
    """Solves B IVPs in one segmented launch sequence (precision
    PITN_PREC_MIXED_FP32 / PITN_PREC_FP64_FF: the reduced-precision scans,
    on the per-IVP path).

    Returns (traj [sum N][d], offsets [B+1], iters [B], status [B], res [B]).
    """
    torch = _torch()
    p_t = _as_f64(params, device)
    x0_t = _as_f64(x0, device)
    h_t = _as_f64(h, device)
    N_t = torch.as_tensor(N, dtype=torch.int64).to(device).contiguous()
    B, d = int(x0_t.shape[0]), int(x0_t.shape[1])
    total = int(torch.as_tensor(N, dtype=torch.int64).sum())
    traj = torch.empty((total, d), dtype=torch.float64, device=device)
    offsets = torch.empty(B + 1, dtype=torch.int64, device=device)
    iters = torch.empty(B, dtype=torch.int32, device=device)
    status = torch.empty(B, dtype=torch.int32, device=device)
    res = torch.empty(B, dtype=torch.float64, device=device)
    opt = P.make_options(guard_B=guard_B, stream=_stream_ptr(stream, device), tile_elems=tile_elems,
                         precision=precision)
    rc = P.pitn_solve_batch(system, B, p_t, x0_t, h_t, N_t, d, tol, max_iter, traj, offsets, iters,
                            status, res, opt)
    P.check(rc, "pitn_solve_batch")
    return traj, offsets, iters, status, res


def backward(system, params, x0, h, N, traj, grad_traj=None, grad_xN=None, ckpt_every=1024,
             device="cuda", stream=None):
    """Adjoint gradients (dL/dx0 [B][d], dL/dparams [B][P]) of a loss of the trajectories."""
    torch = _torch()
    p_t = _as_f64(params, device)
    x0_t = _as_f64(x0, device)
    h_t = _as_f64(h, device)
    N_t = torch.as_tensor(N, dtype=torch.int64).to(device).contiguous()
    B, d = int(x0_t.shape[0]), int(x0_t.shape[1])
    npar = P.pitn_num_params(system)
    gx0 = torch.empty((B, d), dtype=torch.float64, device=device)
    gp = torch.empty((B, npar), dtype=torch.float64, device=device)
    gt = grad_traj.contiguous() if grad_traj is not None else None
    gN = grad_xN.contiguous() if grad_xN is not None else None
    opt = P.make_options(stream=_stream_ptr(stream, device))
    rc = P.pitn_backward(system, B, p_t, x0_t, h_t, N_t, d, traj.contiguous(), gt, gN, ckpt_every,
                         gx0, gp, opt)
    P.check(rc, "pitn_backward")
    return gx0, gp
