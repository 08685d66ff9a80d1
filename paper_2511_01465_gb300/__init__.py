"""GB300-native parallel-in-time Newton ODE solver (arXiv 2511.01465).

The solver writes a one-step discretisation of dx/dt = f(x) (explicit,
eq. 3.8, or implicit, eq. 3.15) as the root-finding problem h(xi) = 0 over
all N steps and solves it by
Newton's method, each Newton step being an affine recursion (eq. 3.13)
computed by a parallel prefix scan (eqs. 3.1-3.4).  All computation runs in
the CUDA library ``libpitn.so`` (C ABI: ``include/pitn.h``); this package is
its Python binding.

Modules:
  pitn       ctypes binding, same names as the C ABI
  api        torch helpers: solve, solve_batch, backward
  autograd   torch.autograd.Function over solve_batch/backward (import it explicitly)
  workloads  seeded synthetic inputs
  build      nvcc build of libpitn.so
"""
from . import pitn, workloads  # noqa: F401
from .pitn import (  # noqa: F401
    PITN_OK, PITN_NOT_CONVERGED, PITN_NONFINITE, PITN_EINVAL, PITN_ENOMEM, PITN_ECUDA,
    PITN_ETIMEOUT, PITN_EUNSUPPORTED, PITN_LORENZ63, PITN_VDP, PITN_LINEAR_OSC, PITN_FKPP,
    PITN_LOGISTIC, PITN_DAHLQUIST, PITN_ROBERTSON, PITN_STEP_EULER, PITN_STEP_RK4,
    PITN_STEP_BACKWARD_EULER, PITN_STEP_TRAPEZOID,
    PITN_PREC_FP64, PITN_PREC_MIXED_BF16, PITN_PREC_MIXED_FP32, PITN_PREC_FP64_FF, PITN_PREC_MIXED_TF32, PitnError, pitn_solve, pitn_solve_ex, pitn_solve_batch,
    pitn_backward, pitn_status_string, pitn_release_workspace, pitn_launch_count, pitn_num_params,
)
from .api import solve, solve_batch, backward  # noqa: F401
