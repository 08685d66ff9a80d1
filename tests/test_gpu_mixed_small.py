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
