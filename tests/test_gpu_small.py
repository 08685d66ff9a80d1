"""GPU parity of the small-state Newton path (d = 2, 3) against the CPU oracle.

Element-wise comparison of trajectories (max relative error, normalised by
the largest reference entry, <= 1e-10 for the FP64 path), bit-exact
comparison of the integer outcomes (Newton updates, status, guard index,
the guard cut of every Newton step) wherever they are fixed by the
mathematics; guarded solves whose guard cuts are held to the spread that
rounding alone produces, measured on the oracle's rounding variants
(tests/rounding.py).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import rounding as R
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL = 1e-10
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_full_size.json")
SPREAD = os.path.join(os.path.dirname(__file__), "golden", "oracle_rounding_spread.json")


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run(pk, wl, tol, max_iter, guard_B=0.0, **kw):
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, max_iter, guard_B=guard_B,
                          history=True, **kw)
    return traj.cpu().numpy(), info


def check_guarded(wl, g, gi, ref, window, first_div, first_res_div, tol):
    """Guarded Newton (reading R8): where the guard cuts, the cut index is
    decided by FP64 comparisons on corrections beyond the converged prefix,
    which grow exponentially there, so the count of updates depends on
    rounding.  The bar is the spread that rounding alone produces, measured
    on the oracle's rounding variants (tests/rounding.py): the status equal,
    the count within the variants' window of the oracle's, the cuts and the
    residual history equal up to the first step at which a variant cut
    elsewhere, the residual history equal until rounding alone moves it.
    Then what is unique: the root of a converged solve, and for a
    capped solve the prefix invariant (the first `iters` states are exact)
    and the guard fill."""
    R.check_guarded(gi["status"], gi["iters"], gi["cut_history"], gi["res_history"], ref, window,
                    first_div, first_res_div)
    if ref["status"] == O.OK:
        assert gi["final_res"] <= tol
        seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
        assert relerr(g, seq) <= TOL_REL
    elif ref["status"] == O.NOT_CONVERGED:
        seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
        k = gi["iters"]
        assert relerr(g[:k], seq[:k]) <= TOL_REL
        q = gi["guard_index"]
        assert 0 < q <= wl.N
        if q < wl.N:
            assert np.array_equal(g[q:], np.broadcast_to(g[q - 1], g[q:].shape))


def check_against_oracle(pk, wl, tol, max_iter, guard_B=0.0, **kw):
    g, gi = run(pk, wl, tol, max_iter, guard_B, **kw)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, max_iter, guard_B=guard_B)
    cut_seen = (gi["cut_history"] < wl.N).any() or (o["cuts"] < wl.N).any()
    if guard_B > 0 and cut_seen:
        rs = R.runs(wl, tol, max_iter, guard_B)
        window, first_div, first_res_div = R.spread(rs)
        check_guarded(wl, g, gi, rs[None], window, first_div, first_res_div, tol)
        return g, gi, o
    assert gi["iters"] == o["iters"]
    assert gi["status"] == o["status"]
    assert gi["guard_index"] == o["guard_index"]
    assert np.array_equal(gi["cut_history"], o["cuts"])
    assert relerr(g, o["traj"]) <= TOL_REL
    np.testing.assert_allclose(gi["res_history"], o["res_hist"], rtol=1e-6, atol=1e-13)
    return g, gi, o


def load_gold():
    with open(GOLD) as f:
        return json.load(f)


def load_spread():
    with open(SPREAD) as f:
        d = json.load(f)
    for v in d.values():
        if isinstance(v, dict):
            v["oracle"]["res_hist"] = v["oracle"]["res_history"]
    return d


FULL = {
    "lorenz_8192_plain_tol1e-10_it50": W.lorenz(),
    "lorenz_8192_guard100_tol1e-10_it50": W.lorenz(),
    "lorenz_8192_guard100_tol1e-12_it100": W.lorenz(),
    "vdp_2^22_plain_tol1e-8_it200": W.vdp(),
    "vdp_2^22_guard100_tol1e-12_it400": W.vdp(),
    "osc_2^22_plain_tol1e-8_it10": W.damped_oscillator(),
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_against_oracle(pk, name):
    """Full-size workloads: integer outcomes equal the oracle's stored ones,
    residual histories agree, converged trajectories equal the sequential
    integration (the unique root of eq. 3.8)."""
    gold = load_gold()[name]
    wl = FULL[name]
    g, gi = run(pk, wl, gold["tol"], gold["max_iter"], gold["guard_B"])
    if gold["guard_B"] > 0:
        sp = load_spread()[name]
        assert sp["oracle"]["iters"] == gold["iters"] and sp["oracle"]["status"] == gold["status"]
        check_guarded(wl, g, gi, sp["oracle"], sp["window"], sp["first_div"], sp["first_res_div"],
                      gold["tol"])
        return
    assert (gi["iters"], gi["status"], gi["guard_index"]) == \
        (gold["iters"], gold["status"], gold["guard_index"])
    np.testing.assert_allclose(gi["res_history"], gold["res_history"], rtol=1e-6, atol=1e-13)
    if gold["status"] == O.OK:
        seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
        assert relerr(g, seq) <= TOL_REL
    elif wl.N <= 1 << 16:
        o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, gold["tol"], gold["max_iter"],
                     guard_B=gold["guard_B"])
        assert relerr(g, o["traj"]) <= TOL_REL


SIZES = [1, 2, 3, 31, 32, 33, 255, 256, 257, 1000, 4097, 20011]


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("kind", ["vdp", "lorenz_plain", "lorenz_guard", "osc"])
def test_ragged_sizes(pk, N, kind):
    if kind == "vdp":
        wl, B = W.vdp(N=N, h=1e-3), 0.0
    elif kind == "lorenz_plain":
        wl, B = W.lorenz(N=N), 0.0
    elif kind == "lorenz_guard":
        wl, B = W.lorenz(N=N), 100.0
    else:
        wl, B = W.damped_oscillator(N=N, h=1e-3), 0.0
    check_against_oracle(pk, wl, 1e-10, 80, B)


@pytest.mark.parametrize("C", [2, 4, 8])
def test_tile_shapes_agree(pk, C):
    wl = W.vdp(N=30001, h=1e-3)
    check_against_oracle(pk, wl, 1e-10, 60, 0.0, tile_elems=C)


def test_prefix_exactness_after_k_updates(pk):
    wl = W.vdp(N=5000, h=1e-2)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    rng = np.random.default_rng(3)
    guess = rng.normal(0, 1, (wl.N, 2))
    for k in (1, 2, 3, 7):
        g, gi = run(pk, wl, 0.0, k, guard_B=1e6, guess=guess)
        assert gi["iters"] == k
        np.testing.assert_allclose(g[:k], seq[:k], rtol=1e-13, atol=1e-13)
        o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, k, guard_B=1e6, guess=guess)
        assert gi["guard_index"] == o["guard_index"]
        # far from the root (random guess, corrections up to 1e5) rounding is
        # amplified through the products of Jacobians over thousands of steps;
        # the prefix above is the unique part, the rest agrees to 1e-8
        assert relerr(g, o["traj"]) <= 1e-8


def test_max_iter_zero_evaluates_residual_only(pk):
    wl = W.lorenz(N=1000)
    g, gi = run(pk, wl, 1e-10, 0)
    assert gi["iters"] == 0 and gi["status"] == O.NOT_CONVERGED
    assert gi["res_history"][0] == pytest.approx(0.026, rel=1e-14)
    assert np.array_equal(g, np.broadcast_to(wl.x0, g.shape))


def test_nonfinite_initial_value(pk):
    wl = W.vdp(N=100)
    wl.x0 = np.array([np.nan, 0.0])
    g, gi = run(pk, wl, 1e-10, 5)
    assert gi["status"] == O.NONFINITE and gi["iters"] == 0


def test_host_pointers_and_guess(pk):
    """The C ABI takes host arrays too (staged through device memory)."""
    from paper_2511_01465_gb300 import pitn as P
    wl = W.lorenz(N=777)
    out = np.zeros((wl.N, 3))
    guess = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N) + 1e-3
    opt = P.make_options(guard_B=100.0, guess=guess)
    rc, res = P.pitn_solve_ex(wl.system, wl.params, wl.x0, wl.h, wl.N, 3, 1e-10, 40, out, opt)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 40, guard_B=100.0, guess=guess)
    assert rc == o["status"] == O.OK and res.iters == o["iters"]
    assert relerr(out, o["traj"]) <= TOL_REL
    rc = P.pitn_solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 3, 1e-10, 40, out)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 40)
    assert rc == o["status"]
    assert relerr(out, o["traj"]) <= TOL_REL


def test_deterministic(pk):
    wl = W.vdp(N=100003, h=1e-3)
    a, ia = run(pk, wl, 1e-10, 40)
    b, ib = run(pk, wl, 1e-10, 40)
    assert np.array_equal(a, b)
    for key in ("iters", "status", "guard_index", "final_res"):
        assert ia[key] == ib[key]
    assert np.array_equal(ia["res_history"], ib["res_history"])
    # guarded regime: counts depend on rounding order, so repeatability matters
    wl = W.lorenz()
    a, ia = run(pk, wl, 1e-12, 100, guard_B=100.0)
    b, ib = run(pk, wl, 1e-12, 100, guard_B=100.0)
    assert np.array_equal(a, b) and ia["iters"] == ib["iters"]


def test_one_launch_per_solve(pk):
    wl = W.vdp(N=65536, h=1e-3)
    before = pk.pitn_launch_count()
    run(pk, wl, 1e-10, 40)
    assert pk.pitn_launch_count() - before == 1
