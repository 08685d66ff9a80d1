"""The allocation-free entry point pitn_solve_noalloc, called through the C ABI.

It exists for callers that may not allocate device memory while running
(real-time control loops, hosts whose allocator owns the device memory): its
scratch is a fixed __device__ array inside the library.  Its results must
equal those of the workspace-backed pitn_solve_ex on the same inputs, for
two calls in a row (the second finds the array holding the first call's
contents).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL_REL = 1e-10


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_01465_gb300 import pitn
    # the allocation-free solve always takes the default launch shape: make
    # the workspace-backed solve take it too, whatever ran before
    pitn.pitn_tune_enable(False)
    pitn.pitn_tune_clear()
    return pitn


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def both(P, wl, tol, max_iter, guard_B):
    dev = torch.device("cuda", 0)
    p = torch.tensor(wl.params, dtype=torch.float64, device=dev)
    x0 = torch.tensor(wl.x0, dtype=torch.float64, device=dev)
    ref = torch.empty((wl.N, wl.d), dtype=torch.float64, device=dev)
    rc_ref, r_ref = P.pitn_solve_ex(wl.system, p, x0, wl.h, wl.N, wl.d, tol, max_iter, ref,
                                    P.make_options(guard_B=guard_B))
    out = torch.full((wl.N, wl.d), float("nan"), dtype=torch.float64, device=dev)
    rc, r = P.pitn_solve_noalloc(wl.system, p, x0, wl.h, wl.N, wl.d, tol, max_iter, guard_B, out)
    torch.cuda.synchronize()
    return (rc_ref, r_ref, ref.cpu().numpy()), (rc, r, out.cpu().numpy())


CASES = [
    (W.vdp(N=30001, h=1e-3), 1e-10, 60, 0.0),
    (W.lorenz(N=8192), 1e-12, 100, 100.0),
    (W.damped_oscillator(N=65536, h=1e-3), 1e-10, 5, 0.0),
    (W.lorenz(N=777), 1e-10, 40, 0.0),
]


def test_noalloc_matches_workspace_solve_twice(P):
    for _ in range(2):  # two calls in a row per case
        for wl, tol, it, B in CASES:
            (rc_ref, r_ref, ref), (rc, r, out) = both(P, wl, tol, it, B)
            assert rc == rc_ref
            assert (r.iters, r.status, r.guard_index) == (r_ref.iters, r_ref.status, r_ref.guard_index)
            assert r.final_res == pytest.approx(r_ref.final_res, rel=1e-12, abs=0.0)
            assert relerr(out, ref) <= TOL_REL


def check_same(P, case):
    (rc_ref, r_ref, ref), (rc, r, out) = both(P, *case)
    assert rc == rc_ref
    assert (r.iters, r.status, r.guard_index) == (r_ref.iters, r_ref.status, r_ref.guard_index)
    assert r.final_res == pytest.approx(r_ref.final_res, rel=1e-12, abs=0.0)
    assert relerr(out, ref) <= TOL_REL
    return r


def test_noalloc_full_iteration_budget_then_a_fresh_solve(P):
    """A solve that uses all of the array's per-iteration records, then
    normal solves at once: they must start clean although the array holds
    the first call's barrier words, error word, record and residual history.
    A guard bound below every correction cuts each Newton step at its first
    state, so the iterate never moves and the solve runs its whole budget of
    1024 updates, whatever the rounding."""
    r = check_same(P, (W.lorenz(N=4096), 1e-10, 1024, 1e-300))
    assert r.status == P.PITN_NOT_CONVERGED and r.iters == 1024 and r.guard_index == 0
    check_same(P, (W.vdp(N=30001, h=1e-3), 1e-10, 60, 0.0))
    check_same(P, (W.lorenz(N=777), 1e-10, 40, 0.0))


def test_noalloc_rejects_sizes_beyond_its_array(P):
    dev = torch.device("cuda", 0)
    wl = W.vdp(N=65537, h=1e-3)
    out = torch.empty((wl.N, 2), dtype=torch.float64, device=dev)
    rc, _ = P.pitn_solve_noalloc(wl.system, wl.params, wl.x0, wl.h, wl.N, 2, 1e-10, 10, 0.0, out)
    assert rc == P.PITN_EINVAL
    wl = W.vdp(N=100, h=1e-3)
    out = torch.empty((wl.N, 2), dtype=torch.float64, device=dev)
    rc, _ = P.pitn_solve_noalloc(wl.system, wl.params, wl.x0, wl.h, wl.N, 2, 1e-10, 1025, 0.0, out)
    assert rc == P.PITN_EINVAL
    # a host trajectory cannot be staged without allocating
    rc, _ = P.pitn_solve_noalloc(wl.system, wl.params, wl.x0, wl.h, wl.N, 2, 1e-10, 10, 0.0,
                                 np.zeros((wl.N, 2)))
    assert rc == P.PITN_EINVAL
