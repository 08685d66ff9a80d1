"""The classical RK4 step map (eq. 2.3) on the GPU path: the paper's printed
Newton residual traces (Sec. 4.1, logistic and van der Pol, delta t = 1e-2,
guess ones) reproduced by the CUDA kernels, and parity with the oracle."""
import json
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_residual_traces.json")


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


SYS = {"logistic": 5, "van_der_pol": 2}


@pytest.mark.parametrize("key", ["logistic", "van_der_pol"])
def test_gpu_reproduces_paper_residual_trace(pk, key):
    with open(GOLD) as f:
        g = json.load(f)[key]
    N, d = g["N"], len(g["x0"])
    guess = np.full((N, d), g["guess"])
    traj, info = pk.solve(SYS[key], g["params"], g["x0"], g["h"], N, 2e-14, 30, guess=guess,
                          history=True, method=pk.PITN_STEP_RK4)
    paper = np.array(g["residuals"])
    assert info["status"] == pk.PITN_OK
    assert info["iters"] + 1 == g["K"] == len(paper)
    for k, (a, b) in enumerate(zip(info["res_history"], paper)):
        assert abs(a - b) <= 1e-8 * abs(b) + 1e-15, (k, a, b)


@pytest.mark.parametrize("key", ["logistic", "van_der_pol"])
@pytest.mark.parametrize("N", [1, 7, 1000, 20001])
def test_rk4_against_oracle(pk, key, N):
    with open(GOLD) as f:
        g = json.load(f)[key]
    d = len(g["x0"])
    guess = np.full((N, d), g["guess"])  # the paper's initial guess (plain Newton converges from it)
    traj, info = pk.solve(SYS[key], g["params"], g["x0"], g["h"], N, 1e-12, 40, history=True,
                          method=pk.PITN_STEP_RK4, guess=guess)
    o = O.newton(SYS[key], g["params"], g["x0"], g["h"], N, 1e-12, 40, method=O.RK4, guess=guess)
    assert (info["iters"], info["status"]) == (o["iters"], o["status"])
    t = traj.cpu().numpy()
    assert np.abs(t - o["traj"]).max() <= 1e-10 * np.abs(o["traj"]).max()


def test_logistic_euler_against_oracle(pk):
    traj, info = pk.solve(5, [1.0, 1.0], [0.1], 1e-3, 10000, 1e-12, 40, history=True)
    o = O.newton(O.LOGISTIC, [1.0, 1.0], [0.1], 1e-3, 10000, 1e-12, 40)
    assert (info["iters"], info["status"]) == (o["iters"], o["status"])
    assert np.abs(traj.cpu().numpy() - o["traj"]).max() <= 1e-10
    np.testing.assert_allclose(info["res_history"], o["res_hist"], rtol=1e-6, atol=1e-15)


def test_rk4_unsupported_systems(pk):
    from paper_2511_01465_gb300 import pitn as P
    with pytest.raises(P.PitnError):
        pk.solve(1, [10, 28, 8 / 3], [1, 1, 1], 1e-3, 100, 1e-10, 5, method=pk.PITN_STEP_RK4)


def test_bench_size_vdp_rk4(pk):
    """The RK4 bench workload at full size (Sec. 4.1's van der Pol on [0, 10]
    at h = 1e-5, N = 1e6, guess ones, tol 1e-8): Newton count and status equal
    the oracle's stored outcome, the residual history matches it, and the
    returned trajectory passes the oracle's residual test on its own."""
    from paper_2511_01465_gb300 import workloads as W
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_full_size.json")) as f:
        gold = json.load(f)["vdp_rk4_1e6_ones_tol1e-8_it50"]
    wl = W.vdp_paper(h=1e-5)
    assert (wl.N, wl.h, gold["method"]) == (gold["N"], gold["h"], O.RK4)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, gold["tol"], gold["max_iter"],
                          guess=np.full((wl.N, wl.d), gold["guess"]), history=True,
                          method=pk.PITN_STEP_RK4)
    assert (info["iters"], info["status"]) == (gold["iters"], gold["status"])
    np.testing.assert_allclose(info["res_history"][:-1], gold["res_history"][:-1], rtol=1e-6, atol=1e-15)
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, traj.cpu().numpy(), method=O.RK4)
    assert not nf and res <= gold["tol"]
