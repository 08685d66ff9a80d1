"""The oracle's rounding variants and the measured spread (CPU only).

The variants (tests/rounding.py) must be the same mathematics as the oracle:
on problems whose Newton iteration has no rounding-sensitive decision they
reach the same counts and the same trajectories to rounding; the stored
spread of the guarded full-size workloads must be consistent with its own
data and with the oracle's stored outcomes."""
import json
import os

import numpy as np
import pytest

import oracle as O
import rounding as R
from paper_2511_01465_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("variant", R.VARIANTS)
def test_variant_is_the_same_newton_iteration(variant):
    """Plain Newton on Lorenz-63 (N = 500) and van der Pol (N = 3000): same
    count, status and cut history as the oracle, trajectories within 1e-12."""
    for wl in (W.lorenz(N=500), W.vdp(N=3000, h=1e-3)):
        a = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
        b = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60, variant=variant)
        assert (a["iters"], a["status"], a["guard_index"]) == (b["iters"], b["status"], b["guard_index"])
        assert np.array_equal(a["cuts"], b["cuts"])
        assert np.abs(a["traj"] - b["traj"]).max() <= 1e-12 * np.abs(a["traj"]).max()
        np.testing.assert_allclose(b["res_hist"], a["res_hist"], rtol=1e-6, atol=1e-14)


def test_scan48_variant_is_the_newton_iteration_to_its_precision():
    """The 48-bit-scan variant: plain Newton on Lorenz-63 (N = 500) and van
    der Pol (N = 3000) takes the oracle's count, status and cuts, and its
    root is the oracle's within 1e-12 (the residual and the update stay FP64,
    so the root does not depend on the step's precision); an affine system
    (the damped oscillator) still converges in one update, with a first
    residual after it of the size of 48-bit rounding, not FP64 rounding."""
    for wl in (W.lorenz(N=500), W.vdp(N=3000, h=1e-3)):
        a = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
        b = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60, variant="s48")
        assert (a["iters"], a["status"], a["guard_index"]) == (b["iters"], b["status"], b["guard_index"])
        assert np.array_equal(a["cuts"], b["cuts"])
        assert np.abs(a["traj"] - b["traj"]).max() <= 1e-12 * np.abs(a["traj"]).max()
    wl = W.damped_oscillator(N=4000, h=1e-3)
    a = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, 1)
    b = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, 1, variant="s48")
    scale = np.abs(a["traj"]).max()
    assert a["res_hist"][1] <= 1e-15 * scale
    assert 1e-16 * scale < b["res_hist"][1] <= 2.0 ** -40 * scale
    assert np.abs(a["traj"] - b["traj"]).max() <= 2.0 ** -40 * scale


@pytest.mark.parametrize("variant", ["blk4", "blk64"])
def test_blocked_bracketing_is_the_newton_step(variant):
    """One Newton step from a random guess bracketed in blocks equals the
    sequential recursion to rounding (Lemma 3.1: any bracketing of eq. 3.3
    is the same product), with block boundaries inside and at the end."""
    wl = W.lorenz(N=301)
    guess = np.random.default_rng(4).normal(0, 1, (wl.N, 3))
    a = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, 1, guess=guess)
    b = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 0.0, 1, guess=guess, variant=variant)
    assert np.abs(a["traj"] - b["traj"]).max() <= 1e-11 * np.abs(a["traj"]).max()
    assert not np.array_equal(a["traj"], guess)


def test_cut_history_of_the_oracle():
    """The cut history has one entry per computed Newton step: N for steps
    that cut nothing, the guard index for the last accepted one, and the
    rejected step of a plain solve that ends on a non-finite correction."""
    wl = W.lorenz(N=500)
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
    assert len(r["cuts"]) == r["iters"] and (r["cuts"] == wl.N).all()
    wl = W.lorenz()
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 20, guard_B=100.0)
    assert len(r["cuts"]) == r["iters"] == 20 and r["cuts"][-1] == r["guard_index"]
    assert (r["cuts"] < wl.N).any()
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 50)     # plain: diverges
    assert r["status"] == O.NONFINITE and len(r["cuts"]) == r["iters"] + 1 and r["cuts"][-1] < wl.N


def test_spread_logic():
    rs = {None: dict(iters=10, cuts=np.array([5, 6, 7, 9])),
          "a": dict(iters=12, cuts=np.array([5, 6, 8, 9])),
          "b": dict(iters=9, cuts=np.array([5, 6, 7, 9, 9]))}
    for r in rs.values():
        r["res_hist"] = np.array([1.0, 2.0, 3.0])
    rs["a"]["res_hist"] = np.array([1.0, 2.0, 3.1])
    assert R.spread(rs) == (2, 2, 2)
    assert R.first_difference([1, 2], [1, 2, 3]) == 2


def test_stored_spread_is_consistent():
    with open(os.path.join(HERE, "golden", "oracle_rounding_spread.json")) as f:
        sp = json.load(f)
    with open(os.path.join(HERE, "golden", "oracle_full_size.json")) as f:
        gold = json.load(f)
    names = [k for k in sp if not k.startswith("_")]
    assert names
    for name in names:
        e = sp[name]
        ref = e["oracle"]
        if name in gold:
            assert (ref["iters"], ref["status"], ref["guard_index"]) == \
                (gold[name]["iters"], gold[name]["status"], gold[name]["guard_index"])
        rejected = ref["status"] == O.NONFINITE and len(ref["cuts"]) > ref["iters"]
        assert len(ref["cuts"]) == ref["iters"] + (1 if rejected else 0)
        assert len(ref["res_history"]) == ref["iters"] + 1
        fp64 = {k: v for k, v in e["variants"].items() if k in R.VARIANTS}
        assert e["window"] == max(abs(v["iters"] - ref["iters"]) for v in fp64.values())
        assert e["first_div"] == min(v["first_cut_difference"] for v in fp64.values())
        assert e["first_res_div"] == min(v["first_res_difference"] for v in fp64.values())
        ff = e["ff"]   # the FP64 orders and the 48-bit scan together: a bar no tighter
        assert ff["window"] == max(abs(v["iters"] - ref["iters"]) for v in e["variants"].values())
        assert ff["first_div"] == min(v["first_cut_difference"] for v in e["variants"].values())
        assert ff["first_res_div"] == min(v["first_res_difference"] for v in e["variants"].values())
        assert ff["window"] >= e["window"] and ff["first_div"] <= e["first_div"]
        assert set(e["variants"]) == set(R.VARIANTS) | set(O.SCAN_VARIANTS)
        for v in e["variants"].values():
            assert v["status"] == ref["status"]


def test_spread_of_lorenz_8192_recomputed():
    """The Lorenz entries of the stored spread recomputed from the oracle."""
    with open(os.path.join(HERE, "golden", "oracle_rounding_spread.json")) as f:
        e = json.load(f)["lorenz_8192_guard100_tol1e-8_it100"]
    wl = W.lorenz()
    rs = R.runs(wl, 1e-8, 100, 100.0, scan48=True)
    assert R.spread({k: v for k, v in rs.items() if k != "s48"}) == \
        (e["window"], e["first_div"], e["first_res_div"])
    assert R.spread(rs) == (e["ff"]["window"], e["ff"]["first_div"], e["ff"]["first_res_div"])
