"""torch.autograd.Function over the batched Newton solve and its adjoint.

Forward: pitn_solve_batch (B IVPs, concatenated trajectories [sum N][d]).
Backward: pitn_backward, the reverse-time affine scan over the transposed
Jacobians, returning dL/dparams [B][P] and dL/dx0 [B][d].  By the implicit
function theorem the gradient of the converged trajectory does not depend on
the Newton path, so the backward needs only the trajectory.  Step sizes and
lengths are not differentiated.
"""
from __future__ import annotations

import torch

from . import api
from . import pitn as P


class NewtonODESolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, x0, system, h, N, tol, max_iter, guard_B, ckpt_every, precision):
        traj, offsets, iters, status, res = api.solve_batch(
            system, params.detach(), x0.detach(), h, N, tol, max_iter, guard_B=guard_B,
            device=params.device, precision=precision)
        ctx.save_for_backward(params, x0, traj)
        ctx.system, ctx.h, ctx.N, ctx.ckpt = system, h, N, ckpt_every
        ctx.mark_non_differentiable(offsets, status)
        return traj, offsets, status

    @staticmethod
    def backward(ctx, grad_traj, grad_offsets, grad_status):
        params, x0, traj = ctx.saved_tensors
        gx0, gp = api.backward(ctx.system, params.detach(), x0.detach(), ctx.h, ctx.N, traj,
                               grad_traj=grad_traj.contiguous(), ckpt_every=ctx.ckpt,
                               device=params.device)
        return gp, gx0, None, None, None, None, None, None, None, None


def odesolve(system, params, x0, h, N, tol=1e-10, max_iter=100, guard_B=100.0, ckpt_every=1024,
             precision=P.PITN_PREC_FP64):
    """Differentiable batched solve.  params [B][P] and x0 [B][d] are float64 CUDA
    tensors; returns (traj [sum N][d], offsets [B+1], status [B]).  precision
    selects the forward solve's scan (PITN_PREC_MIXED_FP32 / PITN_PREC_FP64_FF:
    an inexact Newton step converged to the same FP64 residual tolerance); the
    adjoint is FP64 on the returned trajectory either way."""
    if not isinstance(h, torch.Tensor):
        h = torch.as_tensor(h, dtype=torch.float64)
    return NewtonODESolve.apply(params, x0, system, h, N, tol, max_iter, guard_B, ckpt_every, precision)


__all__ = ["NewtonODESolve", "odesolve", "P"]
