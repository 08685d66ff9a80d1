"""The implicit rules of Sec. 3.4 (backward Euler, eq. 2.5, and the
trapezoidal rule) with the implicit Newton step on the GPU path: the paper's
printed implicit residual traces and iteration counts (Sec. 4.2, backward
Euler, zero guess) reproduced by the CUDA kernel, and element-wise parity with
the oracle on the same seeded inputs for both rules."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_implicit_traces.json")
SYS = {"dahlquist": O.DAHLQUIST, "robertson": O.ROBERTSON}


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


def _gold(key):
    with open(GOLD) as f:
        return json.load(f)[key]


@pytest.mark.parametrize("key", ["dahlquist", "robertson"])
def test_gpu_reproduces_paper_implicit_trace(pk, key):
    g = _gold(key)
    N, d = g["N"], len(g["x0"])
    traj, info = pk.solve(SYS[key], g["params"], g["x0"], g["h"], N, 2e-14, 60,
                          guess=np.zeros((N, d)), history=True, method=pk.PITN_STEP_BACKWARD_EULER)
    paper = np.array(g["residuals"])
    assert info["status"] == pk.PITN_OK
    assert info["iters"] + 1 == g["K"] == len(paper)
    for k, (a, b) in enumerate(zip(info["res_history"], paper)):
        assert abs(a - b) <= 1e-8 * abs(b) + 1e-15, (k, a, b)


@pytest.mark.parametrize("key,dt", [("dahlquist", 1e-4), ("robertson", 1e-2), ("robertson", 5e-3)])
def test_gpu_paper_iteration_counts(pk, key, dt):
    # Sec. 4.2 iteration-count figure: K independent of delta t
    g = _gold(key)
    wl = W.dahlquist(h=dt) if key == "dahlquist" else W.robertson(h=dt)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 2e-14, 60,
                          guess=np.zeros((wl.N, wl.d)), method=pk.PITN_STEP_BACKWARD_EULER)
    k_paper = {float(k): v for k, v in g["K_vs_dt"].items()}[dt]
    assert info["status"] == pk.PITN_OK and info["iters"] + 1 == k_paper
    # sampled states against the oracle's sequential backward Euler
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N, method=O.BACKWARD_EULER)
    t = traj.cpu().numpy()
    idx = np.unique(np.linspace(0, wl.N - 1, 257).astype(np.int64))
    scale = np.abs(seq).max(axis=0)
    assert (np.abs(t[idx] - seq[idx]) <= 1e-9 * scale + 1e-15).all()
    if key == "robertson":
        np.testing.assert_allclose(t.sum(axis=1), 1.0, atol=1e-12)   # y1 + y2 + y3 conserved


CASES = [
    # name, system, params, x0, h, N, guess (None = x0), guard B
    ("dahlquist_ragged", O.DAHLQUIST, [-1.0], [1.0], 1e-2, 4001, 0.0, 0.0),
    ("robertson_5000", O.ROBERTSON, [0.04, 3e7, 1e4], [1.0, 0.0, 0.0], 0.1, 5000, 0.0, 0.0),
    ("robertson_ragged_x0", O.ROBERTSON, [0.04, 3e7, 1e4], [1.0, 0.0, 0.0], 0.05, 12347, None, 0.0),
    ("robertson_1", O.ROBERTSON, [0.04, 3e7, 1e4], [1.0, 0.0, 0.0], 0.1, 1, 0.0, 0.0),
    ("vdp_stiff", O.VDP, [10.0], [2.0, 0.0], 1e-2, 3001, None, 100.0),
    ("vdp_plain", O.VDP, [1.0], [2.0, 0.0], 1e-2, 999, None, 0.0),
    ("logistic", O.LOGISTIC, [1.0, 1.0], [0.1], 1e-2, 1000, 1.0, 0.0),
]


@pytest.mark.parametrize("rule", ["backward_euler", "trapezoid"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_implicit_against_oracle(pk, case, rule):
    _, sys, p, x0, h, N, gv, B = case
    d = len(x0)
    guess = None if gv is None else np.full((N, d), gv)
    m_gpu, m_or = ((pk.PITN_STEP_BACKWARD_EULER, O.BACKWARD_EULER) if rule == "backward_euler"
                   else (pk.PITN_STEP_TRAPEZOID, O.TRAPEZOID))
    traj, info = pk.solve(sys, p, x0, h, N, 1e-12, 80, guard_B=B, guess=guess, history=True,
                          method=m_gpu)
    o = O.newton(sys, p, x0, h, N, 1e-12, 80, guard_B=B, guess=guess, method=m_or)
    assert o["status"] == O.OK
    assert info["status"] == pk.PITN_OK
    if B == 0.0:
        # plain Newton: the same iterates up to rounding, so the same count and trace
        assert info["iters"] == o["iters"]
        # (relative 1e-6 down to the FP64 floor of states of size 1)
        np.testing.assert_allclose(info["res_history"][:-1], o["res_hist"][:-1], rtol=1e-6, atol=1e-15)
    t = traj.cpu().numpy()
    scale = np.abs(o["traj"]).max(axis=0)
    assert (np.abs(t - o["traj"]) <= 1e-9 * scale + 1e-15).all()
    # the returned trajectory satisfies the implicit residual test on its own
    _, res, nf = O.residual(sys, p, x0, h, t, method=m_or)
    assert not nf and res <= 1e-12 * (1 + 1e-6)


def test_explicit_euler_on_stiff_systems(pk):
    # the stiff test systems also run through the explicit map (eq. 2.2);
    # plain Newton from the constant guess diverges on Robertson (the oracle
    # ends NONFINITE too), so the guard is on
    wl = W.robertson(h=1e-4, t_end=1.0)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-13, 400, guard_B=1.0)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-13, 400, guard_B=1.0)
    assert info["status"] == o["status"] == O.OK
    # both solves stop at ||h||_inf <= 1e-13 (absolute), so they agree to that
    # level against the largest state (global measure, R10), not against y2's 1e-5 scale
    t = traj.cpu().numpy()
    assert np.abs(t - o["traj"]).max() <= 1e-10 * np.abs(o["traj"]).max()
    wl = W.dahlquist(h=1e-3, lam=-3.0)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-13, 5)
    ref = (1.0 + wl.h * -3.0) ** np.arange(1, wl.N + 1)
    assert info["iters"] == 1
    # one update from the constant guess 1 adds corrections of size ~1, so the
    # error is absolute (a few ulps of 1): the global relative measure applies
    assert np.abs(traj.cpu().numpy()[:, 0] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_trapezoid_dahlquist_closed_form(pk):
    lam, h, N = -2.5, 0.03, 200
    ref = ((1.0 + 0.5 * h * lam) / (1.0 - 0.5 * h * lam)) ** np.arange(1, N + 1)
    traj, info = pk.solve(O.DAHLQUIST, [lam], [1.0], h, N, 1e-14, 5, guess=np.zeros((N, 1)),
                          method=pk.PITN_STEP_TRAPEZOID)
    assert info["status"] == pk.PITN_OK and info["iters"] == 1   # affine: one update
    np.testing.assert_allclose(traj.cpu().numpy()[:, 0], ref, rtol=1e-12)


def test_implicit_unsupported_combinations(pk):
    from paper_2511_01465_gb300 import pitn as P
    with pytest.raises(P.PitnError):   # no backward Euler instantiation for Lorenz-63
        pk.solve(1, [10, 28, 8 / 3], [1, 1, 1], 1e-3, 100, 1e-10, 5, method=pk.PITN_STEP_BACKWARD_EULER)
    for prec in (pk.PITN_PREC_MIXED_FP32, pk.PITN_PREC_FP64_FF):   # no implicit Lorenz-63, any precision
        with pytest.raises(P.PitnError):
            pk.solve(1, [10, 28, 8 / 3], [1, 1, 1], 1e-3, 100, 1e-10, 5, method=pk.PITN_STEP_BACKWARD_EULER,
                     precision=prec)


def test_bench_size_robertson(pk):
    """The implicit bench workload at full size (backward Euler, h = 1e-4,
    N = 5e6, zero guess, tol 1e-8): Newton count and status equal the oracle's
    stored outcome, the first residuals match its history, and the returned
    trajectory passes the implicit residual test on its own."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_full_size.json")) as f:
        gold = json.load(f)["robertson_5e6_be_zeros_tol1e-8_it60"]
    wl = W.robertson(h=1e-4)
    assert (wl.N, wl.h) == (gold["N"], gold["h"])
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, gold["tol"], gold["max_iter"],
                          guess=np.zeros((wl.N, wl.d)), history=True, method=pk.PITN_STEP_BACKWARD_EULER)
    assert (info["iters"], info["status"]) == (gold["iters"], gold["status"])
    np.testing.assert_allclose(info["res_history"][:-1], gold["res_history"][:-1], rtol=1e-6, atol=1e-15)
    t = traj.cpu().numpy()
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, t, method=O.BACKWARD_EULER)
    assert not nf and res <= gold["tol"]
    np.testing.assert_allclose(t.sum(axis=1), 1.0, atol=1e-9)   # y1 + y2 + y3 conserved


@pytest.mark.parametrize("rule", ["backward_euler", "trapezoid"])
def test_implicit_singular_step_matrix(pk, rule):
    # 1 - h lam (or 1 - h lam / 2) is exactly 0 at h = 0.5: non-finite
    # residual at the first evaluation, as in the oracle
    m, lam = ((pk.PITN_STEP_BACKWARD_EULER, 2.0) if rule == "backward_euler" else (pk.PITN_STEP_TRAPEZOID, 4.0))
    traj, info = pk.solve(O.DAHLQUIST, [lam], [1.0], 0.5, 20, 1e-12, 10, guess=np.zeros((20, 1)), method=m)
    assert info["status"] == pk.PITN_NONFINITE and info["iters"] == 0


# ---------------------------------------------------------------------------
# The implicit rules with the FP32 delta-form scan (an inexact Newton step):
# the residual M_n^{-1} h_n, the element and the update stay FP64, the
# element's S = J_n - I is rounded to FP32.  It must reach the same FP64 residual
# tolerance, pass the oracle's residual test, and stay within 1e-6 (against
# the largest state) of the FP64 oracle's root; its Newton count is reported,
# not required to match.
# ---------------------------------------------------------------------------
RULES = {"backward_euler": ("PITN_STEP_BACKWARD_EULER", O.BACKWARD_EULER),
         "trapezoid": ("PITN_STEP_TRAPEZOID", O.TRAPEZOID)}


@pytest.mark.parametrize("rule", list(RULES))
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_implicit_fp32_scan(pk, case, rule):
    _, sys, p, x0, h, N, gv, B = case
    d = len(x0)
    guess = None if gv is None else np.full((N, d), gv)
    m_gpu, m_or = getattr(pk, RULES[rule][0]), RULES[rule][1]
    traj, info = pk.solve(sys, p, x0, h, N, 1e-12, 150, guard_B=B, guess=guess, history=True,
                          method=m_gpu, precision=pk.PITN_PREC_MIXED_FP32)
    o = O.newton(sys, p, x0, h, N, 1e-12, 150, guard_B=B, guess=guess, method=m_or)
    assert o["status"] == O.OK
    assert info["status"] == pk.PITN_OK and info["final_res"] <= 1e-12
    t = traj.cpu().numpy()
    _, res, nf = O.residual(sys, p, x0, h, t, method=m_or)
    assert not nf and res <= 1e-12 * (1 + 1e-6)
    assert np.abs(t - o["traj"]).max() <= 1e-6 * np.abs(o["traj"]).max()


def test_bench_size_robertson_fp32_scan(pk):
    """The implicit bench workload (backward Euler, h = 1e-4, N = 5e6, zero
    guess, tol 1e-8) with the FP32 scan: converged, its returned trajectory
    passing the oracle's implicit residual test, the linear invariant
    y1 + y2 + y3 = 1 of the exact root kept to the residual's level."""
    wl = W.robertson(h=1e-4)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-8, 60, guess=np.zeros((wl.N, wl.d)),
                          history=True, method=pk.PITN_STEP_BACKWARD_EULER, precision=pk.PITN_PREC_MIXED_FP32)
    assert info["status"] == pk.PITN_OK and info["final_res"] <= 1e-8
    t = traj.cpu().numpy()
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, t, method=O.BACKWARD_EULER)
    assert not nf and res <= 1e-8 * (1 + 1e-6)
    assert np.abs(t.sum(axis=1) - 1.0).max() <= 1e-6


# ---------------------------------------------------------------------------
# The implicit rules with the float-float scan: the FP64 residual and element,
# the dense folds, scans and replay in pairs of floats (~2^-47).  It must meet
# the FP64 path's bars: plain Newton counts and residual traces equal to the
# oracle's, the root within 1e-9 of the oracle's per component scale, the
# oracle's residual test passed.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("rule", list(RULES))
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_implicit_ff_scan(pk, case, rule):
    _, sys, p, x0, h, N, gv, B = case
    d = len(x0)
    guess = None if gv is None else np.full((N, d), gv)
    m_gpu, m_or = getattr(pk, RULES[rule][0]), RULES[rule][1]
    traj, info = pk.solve(sys, p, x0, h, N, 1e-12, 80, guard_B=B, guess=guess, history=True,
                          method=m_gpu, precision=pk.PITN_PREC_FP64_FF)
    o = O.newton(sys, p, x0, h, N, 1e-12, 80, guard_B=B, guess=guess, method=m_or)
    assert o["status"] == O.OK
    assert info["status"] == pk.PITN_OK
    if B == 0.0:
        assert info["iters"] == o["iters"]
        np.testing.assert_allclose(info["res_history"][:-1], o["res_hist"][:-1], rtol=1e-6, atol=1e-15)
    t = traj.cpu().numpy()
    scale = np.abs(o["traj"]).max(axis=0)
    assert (np.abs(t - o["traj"]) <= 1e-9 * scale + 1e-15).all()
    _, res, nf = O.residual(sys, p, x0, h, t, method=m_or)
    assert not nf and res <= 1e-12 * (1 + 1e-6)


def test_bench_size_robertson_ff_scan(pk):
    """The implicit bench workload with the float-float scan: the oracle's
    stored count and status, its residual history, the residual test and
    the conservation of y1 + y2 + y3 as for the FP64 solve."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_full_size.json")) as f:
        gold = json.load(f)["robertson_5e6_be_zeros_tol1e-8_it60"]
    wl = W.robertson(h=1e-4)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, gold["tol"], gold["max_iter"],
                          guess=np.zeros((wl.N, wl.d)), history=True, method=pk.PITN_STEP_BACKWARD_EULER,
                          precision=pk.PITN_PREC_FP64_FF)
    assert (info["iters"], info["status"]) == (gold["iters"], gold["status"])
    np.testing.assert_allclose(info["res_history"][:-1], gold["res_history"][:-1], rtol=1e-6, atol=1e-15)
    t = traj.cpu().numpy()
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, t, method=O.BACKWARD_EULER)
    assert not nf and res <= gold["tol"]
    np.testing.assert_allclose(t.sum(axis=1), 1.0, atol=1e-9)
