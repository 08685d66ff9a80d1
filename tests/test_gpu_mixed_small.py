"""The small-state solve with its scan in FP32 delta form (an inexact Newton
step; residual, stopping test and update in FP64): it must reach the same
FP64 residual tolerance and stay within 1e-6 of the FP64 oracle's root; its
Newton count is reported, not required to match."""
import numpy as np
import pytest

import oracle as O
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


CASES = [
    ("vdp_2^16", W.vdp(N=1 << 16), 100.0),
    # plain Newton diverges here (the oracle ends NONFINITE too): guarded
    ("vdp_ragged", W.vdp(N=20011, h=1e-3), 100.0),
    ("lorenz_8192", W.lorenz(), 100.0),
    ("lorenz_500_plain", W.lorenz(N=500), 0.0),
    ("osc", W.damped_oscillator(N=30000, h=1e-3), 0.0),
    ("vdp_1", W.vdp(N=1), 0.0),
]


@pytest.mark.parametrize("name,wl,B", CASES, ids=[c[0] for c in CASES])
def test_mixed_small_within_1e6(pk, name, wl, B):
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-11, 400, guard_B=B,
                          precision=pk.PITN_PREC_MIXED_FP32, history=True)
    assert info["status"] == O.OK and info["final_res"] <= 1e-11
    g = traj.cpu().numpy()
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, g)
    assert not nf and res <= 1e-11 * (1 + 1e-6)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    err = float(np.abs(g - seq).max() / np.abs(seq).max())
    assert err <= 1e-6, err


def test_mixed_small_rejects_other_systems(pk):
    from paper_2511_01465_gb300 import pitn as P
    wl = W.fkpp(d=64, N=10)
    with pytest.raises(P.PitnError):
        pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-8, 5, precision=P.PITN_PREC_MIXED_FP32)


def test_bench_size_vdp_mixed(pk):
    """The FP32-scan bench workload at full size (van der Pol N = 2^22, guard
    B = 100, tol 1e-8): converged to the FP64 tolerance, its FP64 residual
    re-checked by the oracle, within 1e-6 of the sequential FP64 trajectory."""
    wl = W.vdp()
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-8, 400, guard_B=100.0,
                          precision=pk.PITN_PREC_MIXED_FP32)
    assert info["status"] == O.OK and info["final_res"] <= 1e-8
    g = traj.cpu().numpy()
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, g)
    assert not nf and res <= 1e-8 * (1 + 1e-6)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    assert float(np.abs(g - seq).max() / np.abs(seq).max()) <= 1e-6


# ---------------------------------------------------------------------------
# The RK4 map (eq. 2.3) with the FP32 delta-form scan: S = J - I from the
# stage chain rule in FP32, the residual the FP64 one.  Sec. 4.1's van der
# Pol from the ones guess on ragged sizes and at the bench size: the FP64
# tolerance reached, the oracle's residual re-check passed, the root within
# 1e-6 of the sequential FP64 RK4 trajectory.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 7, 1000, 4099, 10007])
def test_mixed_rk4_within_1e6(pk, N):
    wl = W.vdp_paper(h=1e-3, t_end=N * 1e-3)
    assert wl.N == N
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, N, 1e-11, 60, guess=np.ones((N, wl.d)),
                          method=pk.PITN_STEP_RK4, precision=pk.PITN_PREC_MIXED_FP32, history=True)
    assert info["status"] == O.OK and info["final_res"] <= 1e-11
    g = traj.cpu().numpy()
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, g, method=O.RK4)
    assert not nf and res <= 1e-11 * (1 + 1e-6)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, N, method=O.RK4)
    assert float(np.abs(g - seq).max() / np.abs(seq).max()) <= 1e-6


def test_mixed_rk4_rejects_other_systems(pk):
    from paper_2511_01465_gb300 import pitn as P
    wl = W.lorenz(N=100)
    with pytest.raises(P.PitnError):
        pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-8, 5, method=P.PITN_STEP_RK4,
                 precision=P.PITN_PREC_MIXED_FP32)


def test_bench_size_vdp_rk4_mixed(pk):
    """The RK4 bench workload (h = 1e-5, N = 1e6, guess ones) with the FP32
    scan.  At the bench's tol 1e-8: converged, its residual re-checked by the
    oracle.  That tolerance still leaves an iterate ~5e-6 (relative) from the
    sequential trajectory after 1e6 steps, the FP64 solve's as well (its last
    residual 6.6e-10, the FP32 solve's 7.1e-9, both after 7 updates), so the
    distance to the sequential FP64 RK4 trajectory is checked at tol 1e-11:
    within 1e-9 (both solves ~5e-12 there)."""
    wl = W.vdp_paper(h=1e-5)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N, method=O.RK4)
    for tol, bar in ((1e-8, None), (1e-11, 1e-9)):
        traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, 50, guess=np.ones((wl.N, wl.d)),
                              method=pk.PITN_STEP_RK4, precision=pk.PITN_PREC_MIXED_FP32)
        assert info["status"] == O.OK and info["final_res"] <= tol
        g = traj.cpu().numpy()
        _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, g, method=O.RK4)
        assert not nf and res <= tol * (1 + 1e-6)
        if bar is not None:
            assert float(np.abs(g - seq).max() / np.abs(seq).max()) <= bar
