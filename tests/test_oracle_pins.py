"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, dense linear algebra, finite differences, exact
integer arithmetic or textbook formulas typed in by hand.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2511_01465_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_residual_traces.json")


def _load_gold():
    with open(GOLD) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Printed values (Sec. 4.1 residual figure): RK4, delta t = 1e-2, guess ones.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("key,sys", [("logistic", O.LOGISTIC), ("van_der_pol", O.VDP)])
def test_paper_residual_trace(key, sys):
    g = _load_gold()[key]
    N, d = g["N"], len(g["x0"])
    guess = np.full((N, d), g["guess"])
    # tolerance inside the bracket the paper's traces imply for its own stop rule
    r = O.newton(sys, g["params"], g["x0"], g["h"], N, 2e-14, 30, guess=guess, method=O.RK4)
    ours = r["res_hist"]
    paper = np.array(g["residuals"])
    assert r["status"] == O.OK
    # paper K = residual evaluations = updates + 1
    assert r["iters"] + 1 == g["K"] == len(paper)
    for k, (a, b) in enumerate(zip(ours, paper)):
        # agreement to rounding: relative 1e-8 until the trace reaches the FP64 floor
        assert abs(a - b) <= 1e-8 * abs(b) + 1e-15, (k, a, b)


def test_first_residual_closed_form():
    # constant guess x_k = x0  =>  h_n = x0 - x0 - h f(x0)  =>  ||h||_inf = h ||f(x0)||_inf
    # Lorenz (1,1,1): f = (0, 1*(28-1)-1, 1-8/3) = (0, 26, -5/3)  -> 0.026 at h=1e-3
    r = O.newton(O.LORENZ63, [10, 28, 8 / 3], [1, 1, 1], 1e-3, 64, 0.0, 0)
    assert r["res_hist"][0] == pytest.approx(0.026, rel=1e-14)
    # Van der Pol (2,0), mu=1: f = (0, mu(1-4)*0 - 2) = (0, -2) -> 2e-4 at h=1e-4
    r = O.newton(O.VDP, [1.0], [2.0, 0.0], 1e-4, 64, 0.0, 0)
    assert r["res_hist"][0] == pytest.approx(2e-4, rel=1e-14)
    assert r["status"] == O.NOT_CONVERGED and r["iters"] == 0


def test_rhs_hand_values():
    # textbook right-hand sides evaluated by hand
    np.testing.assert_allclose(O.rhs(O.LORENZ63, [10, 28, 8 / 3], [1, 2, 3]), [10, 23, 2 - 8], rtol=1e-15)
    np.testing.assert_allclose(O.rhs(O.VDP, [0.5], [2, 3]), [3, 0.5 * (1 - 4) * 3 - 2], rtol=1e-15)
    np.testing.assert_allclose(O.rhs(O.LINEAR_OSC, [2.0, 0.25], [1, 1]), [1, -4 - 1], rtol=1e-15)
    # FKPP d=3: dx=1/4, 1/dx^2=16, D=0.1
    np.testing.assert_allclose(O.rhs(O.FKPP, [0.1], [0.1, 0.2, 0.3]), [0.09, 0.16, -0.43], atol=1e-15)
    np.testing.assert_allclose(O.rhs(O.LOGISTIC, [1.0, 2.0], [0.5]), [0.5 * (1 - 0.25)], rtol=1e-15)


def _fd_jac(fun, x, eps=1e-6):
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for j in range(x.size):
        e = np.zeros_like(x)
        e[j] = eps
        cols.append((fun(x + e) - fun(x - e)) / (2 * eps))
    return np.stack(cols, axis=1)


SYSTEMS = [
    (O.LORENZ63, [10.0, 28.0, 8 / 3], 3),
    (O.VDP, [1.3], 2),
    (O.LINEAR_OSC, [1.7, 0.2], 2),
    (O.FKPP, [1e-3], 7),
    (O.LOGISTIC, [1.0, 2.0], 1),
    (O.DAHLQUIST, [-0.7], 1),
    # Robertson's structure with moderate rate constants: central differences of
    # the quadratic right-hand side stay exact to well inside the tolerance
    (O.ROBERTSON, [0.04, 30.0, 10.0], 3),
]


@pytest.mark.parametrize("sys,p,d", SYSTEMS)
def test_jacobians_match_finite_differences(sys, p, d):
    rng = np.random.default_rng(1)
    x = rng.uniform(-1.5, 1.5, d)
    J = O.rhs_jac(sys, p, x)
    Jfd = _fd_jac(lambda y: O.rhs(sys, p, y), x)
    np.testing.assert_allclose(J, Jfd, rtol=1e-7, atol=1e-7)
    G = O.rhs_dparam(sys, p, x)
    Gfd = _fd_jac(lambda q: O.rhs(sys, q, x), np.array(p, dtype=float)).reshape(d, len(p))
    np.testing.assert_allclose(G, Gfd, rtol=1e-7, atol=1e-7)
    for method in (O.EULER, O.RK4):
        _, Jphi, Gphi = O.step(sys, p, 0.05, x, method=method, jac=True, dparam=True)
        Jfd = _fd_jac(lambda y: O.step(sys, p, 0.05, y, method=method)[0], x)
        np.testing.assert_allclose(Jphi, Jfd, rtol=1e-7, atol=1e-8)
        Gfd = _fd_jac(lambda q: O.step(sys, q, 0.05, x, method=method)[0], np.array(p, dtype=float))
        np.testing.assert_allclose(Gphi, Gfd.reshape(d, len(p)), rtol=1e-7, atol=1e-8)


def test_euler_step_is_textbook():
    x = np.array([0.3, -0.7])
    phi, _, _ = O.step(O.VDP, [1.0], 0.1, x)
    np.testing.assert_allclose(phi, x + 0.1 * np.array([x[1], (1 - x[0] ** 2) * x[1] - x[0]]), rtol=1e-15)


# --------------------------------------------------------------------------
# Newton root = sequential trajectory (h(xi) = 0 has the sequential states as
# its unique root since H is unit lower block-bidiagonal).
# --------------------------------------------------------------------------
CASES = [
    ("lorenz_512_plain", W.lorenz(N=512), 0.0),
    ("lorenz_8192_guarded", W.lorenz(N=8192), 100.0),
    ("vdp_4096", W.vdp(N=4096, h=1e-3), 0.0),
    ("osc_4096", W.damped_oscillator(N=4096, h=1e-3), 0.0),
    ("fkpp_16", W.fkpp(d=16, N=2048, h=5e-5), 0.0),
]


def _relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name,wl,B", CASES, ids=[c[0] for c in CASES])
def test_newton_root_equals_sequential(name, wl, B):
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-13, 200, guard_B=B)
    assert r["status"] == O.OK
    # a residual of size tol per step can move the states by about N * tol
    assert _relerr(r["traj"], seq) <= max(1e-12, wl.N * 1e-13 / np.abs(seq).max())
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, r["traj"])
    assert not nf and res <= 1e-13


def test_prefix_exactness_invariant():
    # dx_1 = -h_1 makes x_1 exact after one update; by induction on eq. (3.13)
    # the first k states are exact after k updates, from any guess.
    wl = W.vdp(N=300, h=1e-2)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    rng = np.random.default_rng(3)
    guess = rng.normal(0, 1, (wl.N, 2))
    for k in (1, 2, 3, 5):
        r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, k, guess=guess, guard_B=1e6)
        assert r["iters"] == k
        np.testing.assert_allclose(r["traj"][:k], seq[:k], rtol=1e-13, atol=1e-13)


def test_affine_system_converges_in_one_update():
    # affine step map -> h(xi) is affine -> Newton is exact after one update
    # (the paper's Dahlquist runs show K = 2 residual evaluations)
    wl = W.damped_oscillator(N=4096, h=1e-3)
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 10)
    assert r["status"] == O.OK and r["iters"] == 1


def test_linear_discrete_closed_form():
    # Euler on x' = M x:  x_n = (I + h M)^n x0, via repeated squaring in numpy
    w, z, h = 1.0, 0.05, 1e-3
    M = np.array([[0.0, 1.0], [-w * w, -2 * z * w]])
    x0 = np.array([2.0, 0.0])
    N = 5000
    r = O.newton(O.LINEAR_OSC, [w, z], x0, h, N, 1e-12, 5)
    seq = O.sequential(O.LINEAR_OSC, [w, z], x0, h, N)
    for n in (1, 17, 1000, 4096, 5000):
        ref = np.linalg.matrix_power(np.eye(2) + h * M, n) @ x0
        np.testing.assert_allclose(seq[n - 1], ref, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(r["traj"][n - 1], ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("sys,p,d", SYSTEMS[:4])
def test_newton_step_equals_dense_solve(sys, p, d):
    # eq. (3.10): dxi = -H^{-1} h(xi) with H from eq. (3.9), solved densely,
    # against the oracle's affine recursion of eq. (3.13) (one update).
    N = 6
    rng = np.random.default_rng(7)
    x0 = rng.uniform(-1, 1, d)
    guess = rng.uniform(-1, 1, (N, d))
    h = 0.05
    r, _, _ = O.residual(sys, p, x0, h, guess)
    H = np.zeros((N * d, N * d))
    for i in range(N):
        H[i * d:(i + 1) * d, i * d:(i + 1) * d] = np.eye(d)
        if i > 0:
            _, J, _ = O.step(sys, p, h, guess[i - 1], jac=True)
            H[i * d:(i + 1) * d, (i - 1) * d:i * d] = -J
    dxi = -np.linalg.solve(H, r.reshape(-1))
    out = O.newton(sys, p, x0, h, N, 0.0, 1, guess=guess, guard_B=1e300)
    np.testing.assert_allclose(out["traj"] - guess, dxi.reshape(N, d), rtol=1e-12, atol=1e-13)


def test_scan_exact_on_small_integers():
    # integer elements keep every product exact in FP64: any bracketing of the
    # operator of eq. (3.3) must give bit-identical prefixes (Lemma 3.1), and
    # the brute-force sum z_n = sum_j (A_n..A_{j+1}) c_j must agree exactly.
    rng = np.random.default_rng(11)
    for d in (1, 2, 3):
        N = 14
        A = rng.integers(-2, 3, (N, d, d)).astype(np.float64)
        c = rng.integers(-3, 4, (N, d)).astype(np.float64)
        z = O.affine_scan(A, c)
        A0 = A.copy()
        A0[0] = 0.0
        for n in range(N):
            # brute force
            s = np.zeros(d)
            for j in range(n + 1):
                P = np.eye(d)
                for m in range(j + 1, n + 1):
                    P = A[m] @ P
                s = s + P @ c[j]
            assert np.array_equal(s, z[n])
            # random bracketing of the composition a_n o ... o a_0
            elems = [(A0[m], c[m]) for m in range(n + 1)]
            while len(elems) > 1:
                i = int(rng.integers(0, len(elems) - 1))
                (A1, b1), (A2, b2) = elems[i], elems[i + 1]
                elems[i:i + 2] = [O.combine(A2, b2, A1, b1)]
            assert np.array_equal(elems[0][1], z[n])
            assert not elems[0][0].any()   # a_0 has matrix 0, eq. (3.4)


def test_quadratic_tail():
    # Theorem 1: ||h|| converges quadratically near the root
    g = _load_gold()["van_der_pol"]
    r = O.newton(O.VDP, g["params"], g["x0"], g["h"], g["N"], 2e-14, 30,
                 guess=np.ones((g["N"], 2)), method=O.RK4)
    rh = r["res_hist"]
    for k in (6, 7):
        assert rh[k + 1] <= 10.0 * rh[k] ** 2
        assert math.log(rh[k + 1]) / math.log(rh[k]) > 1.7


def test_plain_newton_diverges_and_guard_recovers():
    wl = W.lorenz(N=8192)
    plain = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 50)
    assert plain["status"] == O.NONFINITE
    # the returned iterate is the last one whose residual was finite
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, plain["traj"])
    assert not nf and res == plain["res_hist"][plain["iters"]]
    # one guarded update: everything from q on is the last updated state
    g1 = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, 1, guard_B=100.0)
    q = g1["guard_index"]
    assert 0 < q < wl.N
    assert np.array_equal(g1["traj"][q:], np.broadcast_to(g1["traj"][q - 1], (wl.N - q, 3)))


def test_adjoint_matches_central_differences():
    sys, mu, x0, h, N = O.VDP, 1.3, np.array([1.5, -0.5]), 1e-2, 300
    target = np.array([1.0, 0.0])

    def loss(p, x):
        tr = O.sequential(sys, p, x, h, N)
        return float(((tr[-1] - target) ** 2).sum())

    tr = O.sequential(sys, [mu], x0, h, N)
    gx0, gp = O.adjoint(sys, [mu], x0, h, tr, grad_xN=2 * (tr[-1] - target))
    eps = 1e-6
    fd_p = (loss([mu + eps], x0) - loss([mu - eps], x0)) / (2 * eps)
    fd_x = [(loss([mu], x0 + e) - loss([mu], x0 - e)) / (2 * eps) for e in np.eye(2) * eps]
    np.testing.assert_allclose(gp, [fd_p], rtol=1e-6)
    np.testing.assert_allclose(gx0, fd_x, rtol=1e-6)


def test_adjoint_with_trajectory_loss():
    sys, p, h, N = O.LORENZ63, np.array([10.0, 28.0, 8 / 3]), 1e-3, 200
    x0 = np.array([1.0, 2.0, 3.0])
    rng = np.random.default_rng(5)
    Wt = rng.normal(0, 1, (N, 3))

    def loss(pp, xx):
        return float((O.sequential(sys, pp, xx, h, N) * Wt).sum())

    tr = O.sequential(sys, p, x0, h, N)
    gx0, gp = O.adjoint(sys, p, x0, h, tr, grad_traj=Wt)
    eps = 1e-6
    fd_p = [(loss(p + e, x0) - loss(p - e, x0)) / (2 * eps) for e in np.eye(3) * eps]
    fd_x = [(loss(p, x0 + e) - loss(p, x0 - e)) / (2 * eps) for e in np.eye(3) * eps]
    np.testing.assert_allclose(gp, fd_p, rtol=1e-6)
    np.testing.assert_allclose(gx0, fd_x, rtol=1e-6)


def test_batch_equals_single_solves():
    bt = W.lorenz_batch(B=6, n_min=100, n_max=700)
    out = O.newton_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, 1e-10, 100, guard_B=100.0)
    assert out["offsets"][0] == 0 and np.array_equal(np.diff(out["offsets"]), bt.N)
    for b in range(bt.B):
        r = O.newton(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b], 1e-10, 100, guard_B=100.0)
        s, e = out["offsets"][b], out["offsets"][b + 1]
        assert np.array_equal(out["traj"][s:e], r["traj"])
        assert out["iters"][b] == r["iters"] and out["status"][b] == r["status"]


# --------------------------------------------------------------------------
# Implicit rule (Sec. 3.4, eqs. 3.15-3.19; Sec. 4.2 experiments).
# --------------------------------------------------------------------------
GOLD_IMPLICIT = os.path.join(os.path.dirname(__file__), "golden", "paper_implicit_traces.json")


def _load_gold_implicit():
    with open(GOLD_IMPLICIT) as f:
        return json.load(f)


IMPLICIT = {"dahlquist": O.DAHLQUIST, "robertson": O.ROBERTSON}


@pytest.mark.parametrize("key", ["dahlquist", "robertson"])
def test_paper_implicit_residual_trace(key):
    g = _load_gold_implicit()[key]
    N, d = g["N"], len(g["x0"])
    r = O.newton(IMPLICIT[key], g["params"], g["x0"], g["h"], N, 2e-14, 60,
                 guess=np.full((N, d), g["guess"]), method=O.BACKWARD_EULER)
    paper = np.array(g["residuals"])
    assert r["status"] == O.OK
    assert r["iters"] + 1 == g["K"] == len(paper)
    for k, (a, b) in enumerate(zip(r["res_hist"], paper)):
        assert abs(a - b) <= 1e-8 * abs(b) + 1e-15, (k, a, b)


@pytest.mark.parametrize("key,dt", [("dahlquist", 1e-2), ("dahlquist", 1e-3), ("dahlquist", 1e-4),
                                    ("robertson", 1e-2)])
def test_paper_implicit_iteration_count(key, dt):
    g = _load_gold_implicit()[key]
    N, d = int(round(g["t_end"] / dt)), len(g["x0"])
    r = O.newton(IMPLICIT[key], g["params"], g["x0"], dt, N, 2e-14, 60,
                 guess=np.zeros((N, d)), method=O.BACKWARD_EULER)
    assert r["status"] == O.OK
    assert r["iters"] + 1 == g["K_vs_dt"][repr(dt) if repr(dt) in g["K_vs_dt"] else str(dt)]


def test_backward_euler_dahlquist_closed_form():
    # backward Euler on y' = lambda y: y_n = (1 - h lambda)^{-n} exactly
    lam, h, N = -2.5, 0.03, 200
    ref = (1.0 / (1.0 - h * lam)) ** np.arange(1, N + 1)
    seq = O.sequential(O.DAHLQUIST, [lam], [1.0], h, N, method=O.BACKWARD_EULER)[:, 0]
    np.testing.assert_allclose(seq, ref, rtol=1e-12)
    r = O.newton(O.DAHLQUIST, [lam], [1.0], h, N, 1e-14, 5, guess=np.zeros((N, 1)),
                 method=O.BACKWARD_EULER)
    assert r["status"] == O.OK and r["iters"] == 1      # affine in xi: one update
    np.testing.assert_allclose(r["traj"][:, 0], ref, rtol=1e-12)


def test_backward_euler_root_and_mass_conservation():
    # x_n - x_{n-1} - h f(x_n) = 0 checked with the right-hand side alone, and
    # y1 + y2 + y3 = 1 (the Robertson rates sum to zero, so every backward
    # Euler state conserves the total)
    p, x0, h, N = [0.04, 3e7, 1e4], np.array([1.0, 0.0, 0.0]), 0.05, 400
    r = O.newton(O.ROBERTSON, p, x0, h, N, 1e-14, 60, guess=np.zeros((N, 3)),
                 method=O.BACKWARD_EULER)
    assert r["status"] == O.OK
    x = r["traj"]
    prev = np.vstack([x0, x[:-1]])
    resid = np.array([x[n] - prev[n] - h * O.rhs(O.ROBERTSON, p, x[n]) for n in range(N)])
    assert np.abs(resid).max() < 1e-12
    np.testing.assert_allclose(x.sum(axis=1), 1.0, atol=1e-13)
    seq = O.sequential(O.ROBERTSON, p, x0, h, N, method=O.BACKWARD_EULER)
    np.testing.assert_allclose(x, seq, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("sys,p,d", [(O.DAHLQUIST, [-3.0], 1), (O.ROBERTSON, [0.04, 3e2, 1e2], 3),
                                     (O.VDP, [2.0], 2)])
def test_implicit_newton_step_equals_dense_solve(sys, p, d):
    # eq. (3.17): dxi = -H^{-1} h(xi), H block lower bidiagonal with diagonal
    # I - h df/dx(x_n) and sub-diagonal -I (eq. 3.16), solved densely
    N, h = 7, 0.05
    rng = np.random.default_rng(11)
    x0 = rng.uniform(0, 1, d)
    guess = rng.uniform(0, 1, (N, d))
    prev = np.vstack([x0, guess[:-1]])
    hv = np.concatenate([guess[n] - prev[n] - h * O.rhs(sys, p, guess[n]) for n in range(N)])
    H = np.zeros((N * d, N * d))
    for i in range(N):
        H[i * d:(i + 1) * d, i * d:(i + 1) * d] = np.eye(d) - h * O.rhs_jac(sys, p, guess[i])
        if i > 0:
            H[i * d:(i + 1) * d, (i - 1) * d:i * d] = -np.eye(d)
    dxi = -np.linalg.solve(H, hv)
    out = O.newton(sys, p, x0, h, N, 0.0, 1, guess=guess, guard_B=1e300, method=O.BACKWARD_EULER)
    np.testing.assert_allclose(out["traj"] - guess, dxi.reshape(N, d), rtol=1e-11, atol=1e-13)


def test_trapezoid_dahlquist_closed_form_and_order():
    # trapezoidal rule on y' = lambda y: y_n = ((1 + h lambda/2) / (1 - h lambda/2))^n,
    # and its global error at t = 1 falls 4x when h halves (second order)
    lam, h, N = -2.5, 0.03, 200
    ref = ((1.0 + 0.5 * h * lam) / (1.0 - 0.5 * h * lam)) ** np.arange(1, N + 1)
    seq = O.sequential(O.DAHLQUIST, [lam], [1.0], h, N, method=O.TRAPEZOID)[:, 0]
    np.testing.assert_allclose(seq, ref, rtol=1e-12)
    r = O.newton(O.DAHLQUIST, [lam], [1.0], h, N, 1e-14, 5, guess=np.zeros((N, 1)), method=O.TRAPEZOID)
    assert r["status"] == O.OK and r["iters"] == 1
    np.testing.assert_allclose(r["traj"][:, 0], ref, rtol=1e-12)
    errs = []
    for n in (50, 100, 200):
        y = O.newton(O.DAHLQUIST, [lam], [1.0], 1.0 / n, n, 1e-14, 5, method=O.TRAPEZOID)["traj"][-1, 0]
        errs.append(abs(y - math.exp(lam)))
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


def test_trapezoid_root_and_mass_conservation():
    p, x0, h, N = [0.04, 3e7, 1e4], np.array([1.0, 0.0, 0.0]), 0.05, 400
    r = O.newton(O.ROBERTSON, p, x0, h, N, 1e-14, 80, guess=np.zeros((N, 3)), method=O.TRAPEZOID)
    assert r["status"] == O.OK
    x = r["traj"]
    prev = np.vstack([x0, x[:-1]])
    resid = np.array([x[n] - prev[n] - 0.5 * h * (O.rhs(O.ROBERTSON, p, prev[n]) + O.rhs(O.ROBERTSON, p, x[n]))
                      for n in range(N)])
    assert np.abs(resid).max() < 1e-12
    np.testing.assert_allclose(x.sum(axis=1), 1.0, atol=1e-13)
    seq = O.sequential(O.ROBERTSON, p, x0, h, N, method=O.TRAPEZOID)
    np.testing.assert_allclose(x, seq, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("sys,p,d", [(O.DAHLQUIST, [-3.0], 1), (O.ROBERTSON, [0.04, 3e2, 1e2], 3),
                                     (O.VDP, [2.0], 2), (O.LOGISTIC, [1.0, 2.0], 1)])
def test_trapezoid_newton_step_equals_dense_solve(sys, p, d):
    # eq. (3.17) with H of eq. (3.16): diagonal I - (h/2) df/dx(x_n),
    # sub-diagonal -(I + (h/2) df/dx(x_{n-1})), solved densely
    N, h = 7, 0.05
    rng = np.random.default_rng(12)
    x0 = rng.uniform(0, 1, d)
    guess = rng.uniform(0, 1, (N, d))
    prev = np.vstack([x0, guess[:-1]])
    hv = np.concatenate([guess[n] - prev[n] - 0.5 * h * (O.rhs(sys, p, prev[n]) + O.rhs(sys, p, guess[n]))
                         for n in range(N)])
    H = np.zeros((N * d, N * d))
    for i in range(N):
        H[i * d:(i + 1) * d, i * d:(i + 1) * d] = np.eye(d) - 0.5 * h * O.rhs_jac(sys, p, guess[i])
        if i > 0:
            H[i * d:(i + 1) * d, (i - 1) * d:i * d] = -np.eye(d) - 0.5 * h * O.rhs_jac(sys, p, guess[i - 1])
    dxi = -np.linalg.solve(H, hv)
    out = O.newton(sys, p, x0, h, N, 0.0, 1, guess=guess, guard_B=1e300, method=O.TRAPEZOID)
    np.testing.assert_allclose(out["traj"] - guess, dxi.reshape(N, d), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("method,lam", [(O.BACKWARD_EULER, 2.0), (O.TRAPEZOID, 4.0)])
def test_implicit_singular_step_matrix(method, lam):
    # h = 0.5: I - dg/dx_n = 1 - h lam (backward Euler) or 1 - h lam / 2
    # (trapezoid) is exactly 0, so the implicit residual is not finite and the
    # solve ends NONFINITE at its first evaluation (reading R9)
    r = O.newton(O.DAHLQUIST, [lam], [1.0], 0.5, 20, 1e-12, 10, guess=np.zeros((20, 1)), method=method)
    assert r["status"] == O.NONFINITE and r["iters"] == 0


def test_oracle_wrapper_checks_buffer_sizes():
    # the C routines read fixed-size buffers: the wrapper refuses short ones and
    # broadcasts a constant guess to every step
    with pytest.raises(ValueError):
        O.newton(O.VDP, [1.0, 2.0], [0.0, 1.0], 1e-2, 10, 1e-10, 5)
    with pytest.raises(ValueError):
        O.newton(O.VDP, [1.0], [0.0, 1.0], 1e-2, 10, 1e-10, 5, guess=np.ones((9, 2)))
    a = O.newton(O.VDP, [1.0], [0.0, 1.0], 1e-2, 50, 1e-12, 30, guess=1.0, method=O.RK4)
    b = O.newton(O.VDP, [1.0], [0.0, 1.0], 1e-2, 50, 1e-12, 30, guess=np.ones((50, 2)), method=O.RK4)
    assert a["iters"] == b["iters"] and np.array_equal(a["traj"], b["traj"])
    with pytest.raises(ValueError):
        O.adjoint(O.VDP, [1.0], [0.0, 1.0], 1e-2, np.zeros((5, 2)), grad_xN=np.ones(3))
