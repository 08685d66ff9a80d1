"""The float-float scan (PITN_PREC_FP64_FF) on the GPU.

Its arithmetic (csrc/ffarith.cuh) against FP64 references: the integer-pipe
split of a double into hi + lo is the hardware rounding of the double to
float (exact ties aside) plus a remainder within 2^-47 relative; sums and
products of float-float values are within 2^-44 of the FP64 results
(normwise).  Its solves against the FP64 oracle, at the FP64 path's bars;
where a guarded solve's cuts depend on rounding, within the spread of the
FP64 rounding variants and the 48-bit-scan variant (tests/rounding.py)."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import rounding as R
from paper_2511_01465_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_01465_gb300", "csrc")


def test_ff_against_fp64(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "ff_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "gpu_helpers", "ff_check.cu")], check=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    f = out.stdout.split()
    counts = dict(zip(f[0::2], map(int, f[1::2])))
    assert counts["checked"] >= 1 << 22
    for k in ("split_hi_bad", "split_err", "split_unnorm", "add_bad", "mul_bad", "special_bad"):
        assert counts[k] == 0, counts


# ---------------------------------------------------------------------------
# The float-float solve (PITN_PREC_FP64_FF) against the FP64 oracle: it must
# meet the FP64 path's bars -- trajectories within 1e-10 of the oracle's,
# integer outcomes equal where they are rounding-robust, guarded solves
# within the spread rounding alone produces, the 48-bit scan's included
# (tests/rounding.py).
# ---------------------------------------------------------------------------
TOL_REL = 1e-10
SPREAD = os.path.join(HERE, "golden", "oracle_rounding_spread.json")


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def ff_solve(pk, wl, tol, max_iter, guard_B):
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, max_iter, guard_B=guard_B,
                          precision=pk.PITN_PREC_FP64_FF, history=True)
    return traj.cpu().numpy(), info


@pytest.mark.parametrize("N", [1, 2, 3, 31, 32, 33, 255, 256, 257, 1000, 4097, 20011, 30001])
@pytest.mark.parametrize("kind", ["vdp", "osc", "lorenz"])
def test_ff_plain_equals_oracle(pk, kind, N):
    """Plain Newton: count, status, the cuts of the accepted steps and the
    residual history equal to the oracle's, trajectory within 1e-10.  (Where
    plain Newton diverges, the index at which the rejected last correction
    overflows is where noise of the size of the scan's rounding, grown
    exponentially beyond the converged prefix, reaches the FP64 range: it
    moves with the scan's precision and is not compared.)"""
    wl = {"vdp": lambda: W.vdp(N=N, h=1e-3), "osc": lambda: W.damped_oscillator(N=N, h=1e-3),
          "lorenz": lambda: W.lorenz(N=N)}[kind]()
    g, gi = ff_solve(pk, wl, 1e-10, 60, 0.0)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
    o1 = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, 1)
    if np.abs(o1["traj"] - wl.x0).max() > np.finfo(np.float32).max:
        # the first Newton correction of plain Newton leaves the float range
        # (Lorenz-63 over 20 time units: |dx| ~ 1e99): the float-float scan
        # overflows there and ends NONFINITE before the first update, where
        # FP64 (range 1.8e308) accepts it and overflows one step later
        assert gi["status"] == o["status"] == O.NONFINITE and gi["iters"] == 0
        assert np.array_equal(g, np.broadcast_to(wl.x0, g.shape))
        return
    assert (gi["iters"], gi["status"], gi["guard_index"]) == (o["iters"], o["status"], o["guard_index"])
    k = o["iters"]
    assert len(gi["cut_history"]) == len(o["cuts"])
    assert np.array_equal(gi["cut_history"][:k], o["cuts"][:k])
    np.testing.assert_allclose(gi["res_history"], o["res_hist"], rtol=1e-6, atol=1e-13)
    assert relerr(g, o["traj"]) <= TOL_REL


def test_ff_guarded_ragged(pk):
    """Guarded van der Pol over 20011 steps at tol 1e-12, where the converged
    iterate is the root to FP64 accuracy (at 1e-10 the oracle's own iterate
    is 3.9e-9 from the sequential trajectory)."""
    wl = W.vdp(N=20011, h=1e-3)
    g, gi = ff_solve(pk, wl, 1e-12, 80, 100.0)
    rs = R.runs(wl, 1e-12, 80, 100.0, scan48=True)
    window, first_div, first_res_div = R.spread(rs)
    R.check_guarded(gi["status"], gi["iters"], gi["cut_history"], gi["res_history"], rs[None], window,
                    first_div, first_res_div)
    if rs[None]["status"] == O.OK:
        assert relerr(g, O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)) <= TOL_REL


@pytest.mark.parametrize("name", ["vdp_2^22_guard100_tol1e-8_it400", "vdp_2^22_guard100_tol1e-12_it400"])
def test_ff_bench_size(pk, name):
    """The bench workload (van der Pol, N = 2^22, guard B = 100): converged,
    within the measured rounding spread of the oracle's count, cuts and
    residuals, its FP64 residual re-checked by the oracle; at tol 1e-12 within
    1e-10 of the sequential FP64 trajectory (the root).  At tol 1e-8 the
    tolerance, not the arithmetic, bounds the distance to the root."""
    with open(SPREAD) as f:
        sp = json.load(f)[name]
    ref = dict(sp["oracle"], res_hist=sp["oracle"]["res_history"])
    wl = W.vdp()
    g, gi = ff_solve(pk, wl, sp["tol"], sp["max_iter"], sp["guard_B"])
    ff = sp["ff"]
    R.check_guarded(gi["status"], gi["iters"], gi["cut_history"], gi["res_history"], ref, ff["window"],
                    ff["first_div"], ff["first_res_div"])
    assert gi["final_res"] <= sp["tol"]
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, g)
    assert not nf and res <= sp["tol"] * (1 + 1e-6)
    if sp["tol"] <= 1e-12:
        assert relerr(g, O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)) <= TOL_REL


@pytest.mark.parametrize("name", ["lorenz_8192_guard100_tol1e-12_it100", "lorenz_8192_guard100_tol1e-10_it50"])
def test_ff_lorenz_guarded_8192(pk, name):
    """Lorenz-63 (d = 3, the three-phase float-float kernel) at N = 8192,
    guarded: status, count, cuts and residual history within the rounding
    spread of the oracle's FP64 variants and its 48-bit-scan variant (the
    float-float scan's precision: on this chaotic horizon the 48-bit scan
    cuts elsewhere from step 39, the FP64 orders from step 41); converged,
    the root to 1e-10; capped, the prefix invariant."""
    with open(SPREAD) as f:
        sp = json.load(f)[name]
    ref = dict(sp["oracle"], res_hist=sp["oracle"]["res_history"])
    wl = W.lorenz()
    g, gi = ff_solve(pk, wl, sp["tol"], sp["max_iter"], sp["guard_B"])
    ff = sp["ff"]
    R.check_guarded(gi["status"], gi["iters"], gi["cut_history"], gi["res_history"], ref, ff["window"],
                    ff["first_div"], ff["first_res_div"])
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    if gi["status"] == O.OK:
        assert relerr(g, seq) <= TOL_REL
    else:
        k = gi["iters"]
        assert relerr(g[:k], seq[:k]) <= TOL_REL


def test_ff_rejects_other_systems(pk):
    from paper_2511_01465_gb300 import pitn as P
    wl = W.robertson(h=1e-3)
    with pytest.raises(P.PitnError):
        pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-8, 5, precision=P.PITN_PREC_FP64_FF)


# ---------------------------------------------------------------------------
# The RK4 map (eq. 2.3) with the float-float scan: the stage chain rule of
# the Jacobian in float-float, the residual the FP64 one.  The paper's
# printed Sec. 4.1 trace for van der Pol, counts equal to the oracle's on
# ragged sizes (plain Newton from the ones guess, rounding-robust), the root
# to 1e-10, and the bench workload's outcome.
# ---------------------------------------------------------------------------
RK4_GOLD = os.path.join(HERE, "golden", "paper_residual_traces.json")


def test_ff_rk4_reproduces_paper_trace(pk):
    with open(RK4_GOLD) as f:
        g = json.load(f)["van_der_pol"]
    N, d = g["N"], len(g["x0"])
    traj, info = pk.solve(2, g["params"], g["x0"], g["h"], N, 2e-14, 30, guess=np.full((N, d), g["guess"]),
                          history=True, method=pk.PITN_STEP_RK4, precision=pk.PITN_PREC_FP64_FF)
    paper = np.array(g["residuals"])
    assert info["status"] == pk.PITN_OK
    assert info["iters"] + 1 == g["K"] == len(paper)
    for k, (a, b) in enumerate(zip(info["res_history"], paper)):
        assert abs(a - b) <= 1e-8 * abs(b) + 1e-15, (k, a, b)


@pytest.mark.parametrize("N", [1, 7, 1000, 20001])
def test_ff_rk4_against_oracle(pk, N):
    with open(RK4_GOLD) as f:
        g = json.load(f)["van_der_pol"]
    d = len(g["x0"])
    guess = np.full((N, d), g["guess"])
    traj, info = pk.solve(2, g["params"], g["x0"], g["h"], N, 1e-12, 40, history=True, guess=guess,
                          method=pk.PITN_STEP_RK4, precision=pk.PITN_PREC_FP64_FF)
    o = O.newton(2, g["params"], g["x0"], g["h"], N, 1e-12, 40, method=O.RK4, guess=guess)
    assert (info["iters"], info["status"]) == (o["iters"], o["status"])
    np.testing.assert_allclose(info["res_history"], o["res_hist"], rtol=1e-6, atol=1e-13)
    assert relerr(traj.cpu().numpy(), o["traj"]) <= TOL_REL


def test_ff_rk4_bench_size(pk):
    """The RK4 bench workload (Sec. 4.1's van der Pol on [0, 10], h = 1e-5,
    N = 1e6, guess ones, tol 1e-8): count and status equal the oracle's stored
    outcome, residual history within 1e-6, the returned trajectory passing the
    oracle's residual test."""
    with open(os.path.join(HERE, "golden", "oracle_full_size.json")) as f:
        gold = json.load(f)["vdp_rk4_1e6_ones_tol1e-8_it50"]
    wl = W.vdp_paper(h=1e-5)
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, gold["tol"], gold["max_iter"],
                          guess=np.full((wl.N, wl.d), gold["guess"]), history=True,
                          method=pk.PITN_STEP_RK4, precision=pk.PITN_PREC_FP64_FF)
    assert (info["iters"], info["status"]) == (gold["iters"], gold["status"])
    np.testing.assert_allclose(info["res_history"][:-1], gold["res_history"][:-1], rtol=1e-6, atol=1e-15)
    _, res, nf = O.residual(wl.system, wl.params, wl.x0, wl.h, traj.cpu().numpy(), method=O.RK4)
    assert not nf and res <= gold["tol"]
