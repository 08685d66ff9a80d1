"""Runs one workload a few times, for profiling under ncu.

    python -m paper_2511_01465_gb300.profile_workload --workload vdp --N 1048576 --max-iter 10 --repeat 2
    ncu --set full --clock-control none -k regex:newton_small -s 1 -c 1 \\
        python -m paper_2511_01465_gb300.profile_workload --workload vdp --N 1048576 --max-iter 10

Workloads: vdp, lorenz, osc (single IVP; --precision 2 for the FP32 delta
scan), vdp_rk4 (RK4 van der Pol on [0, 10], h = 10 / N, from the ones
guess, or from the root with --from-root), robertson (backward Euler from
the zero guess, h = 500 / N; --precision 2 for the FP32 scan), fkpp,
fkpp_mixed, fkpp_tf32 (d = 128; BF16 / TF32 tensor-core composes),
batch (Lorenz batch, --B IVPs of lengths in [--nmin, --nmax]; --precision
2 / 3 for the FP32 / float-float scans), adjoint
(Van der Pol batch forward + backward).  Sizes default to the small cases
used for full captures; prints the outcome of the last repetition.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="vdp")
    ap.add_argument("--N", type=int, default=1 << 20)
    ap.add_argument("--max-iter", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--guard", type=float, default=100.0)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--B", type=int, default=512)
    ap.add_argument("--nmin", type=int, default=1 << 10)
    ap.add_argument("--nmax", type=int, default=1 << 13)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--from-root", action="store_true",
                    help="single-IVP workloads: solve once (tol 1e-12), then time solves that start "
                         "from that root (every Newton pass then covers all N steps)")
    a = ap.parse_args()

    import torch

    from . import api, workloads as W
    from .pitn import (PITN_PREC_FP64, PITN_PREC_MIXED_BF16, PITN_PREC_MIXED_TF32, PITN_STEP_BACKWARD_EULER,
                       PITN_STEP_RK4)

    out = None
    root = None
    for _ in range(a.repeat):
        if a.workload in ("vdp", "lorenz", "osc"):
            wl = {"vdp": W.vdp, "lorenz": W.lorenz, "osc": W.damped_oscillator}[a.workload](N=a.N)
            guess = None
            if a.from_root:
                if root is None:
                    root = api.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-12, 400, guard_B=a.guard)[0]
                guess = root
            out = api.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, a.tol, a.max_iter, guard_B=a.guard,
                            precision=a.precision, guess=guess)[1]
        elif a.workload == "vdp_rk4":
            wl = W.vdp_paper(h=10.0 / a.N)
            guess = np.ones((wl.N, wl.d))
            if a.from_root:
                if root is None:
                    root = api.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-12, 50, guess=guess,
                                     method=PITN_STEP_RK4)[0]
                guess = root
            out = api.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, a.tol, a.max_iter, guess=guess,
                            method=PITN_STEP_RK4)[1]
        elif a.workload == "robertson":
            wl = W.robertson(h=500.0 / a.N)
            out = api.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, a.tol, a.max_iter,
                            guess=np.zeros((wl.N, wl.d)), method=PITN_STEP_BACKWARD_EULER,
                            precision=a.precision)[1]
        elif a.workload in ("fkpp", "fkpp_mixed", "fkpp_tf32"):
            wl = W.fkpp(N=a.N)
            prec = {"fkpp": PITN_PREC_FP64, "fkpp_mixed": PITN_PREC_MIXED_BF16,
                    "fkpp_tf32": PITN_PREC_MIXED_TF32}[a.workload]
            out = api.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, a.tol, a.max_iter, precision=prec)[1]
        elif a.workload == "batch":
            bt = W.lorenz_batch(B=a.B, n_min=a.nmin, n_max=a.nmax)
            r = api.solve_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, a.tol, a.max_iter, guard_B=a.guard,
                                precision=a.precision)
            from .pitn import pitn_batch_work
            out = {"mean_iters": float(r[2].float().mean()), "converged": int((r[3] == 0).sum()),
                   "steps_evaluated_replayed": pitn_batch_work()}
        elif a.workload == "adjoint":
            bt = W.vdp_adjoint_batch(B=a.B, N=a.N)
            traj, offs, it, st, res = api.solve_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, 1e-12,
                                                      a.max_iter, guard_B=a.guard)
            last = offs[1:] - 1
            gN = (2.0 * (traj[last] - torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda"))).contiguous()
            gx0, gp = api.backward(bt.system, bt.params, bt.x0, bt.h, bt.N, traj, grad_xN=gN)
            out = {"grad_norm": float(np.linalg.norm(gp.cpu().numpy()))}
        else:
            raise SystemExit(f"unknown workload {a.workload}")
    torch.cuda.synchronize()
    print(out)


if __name__ == "__main__":
    main()
