"""GPU parity of the batched (segmented) solve against per-IVP oracle solves.

Integer outputs (offsets, Newton counts, statuses) are compared bit-exactly
where the solve is in the rounding-robust regime (plain Newton, or guarded
runs whose guard never cut); guarded runs whose guard cut are checked for
what is unique (status, root, prefix invariant, fill) and for a Newton count
within the spread that rounding alone produces on the oracle's rounding
variants (tests/rounding.py).
"""
import numpy as np
import pytest

import oracle as O
import rounding as R
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL_REL = 1e-10


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run_batch(pk, bt, tol, max_iter, guard_B, tile_elems=0, precision=0):
    traj, offs, iters, status, res = pk.solve_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, tol,
                                                    max_iter, guard_B=guard_B, tile_elems=tile_elems,
                                                    precision=precision)
    return (traj.cpu().numpy(), offs.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy(),
            res.cpu().numpy())


def compare(bt, out, tol, max_iter, guard_B, sample=None):
    traj, offs, iters, status, res = out
    assert offs[0] == 0 and np.array_equal(np.diff(offs), bt.N)
    idx = range(bt.B) if sample is None else sample
    for b in idx:
        s, e = offs[b], offs[b + 1]
        o = O.newton(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b], tol, max_iter,
                     guard_B=guard_B)
        g = traj[s:e]
        assert status[b] == o["status"], b
        robust = guard_B <= 0 or (o["guard_index"] == bt.N[b] and o["iters"] == iters[b])
        if robust:
            assert iters[b] == o["iters"], b
            assert relerr(g, o["traj"]) <= TOL_REL, b
            if o["status"] != O.NONFINITE:
                assert res[b] == pytest.approx(o["res_hist"][o["iters"]], rel=1e-6, abs=1e-13)
        elif o["status"] == O.OK:
            # the guard cut: the count may move by what rounding alone moves it,
            # measured on the oracle's rounding variants for this IVP
            wl = W.Single("ivp", bt.system, bt.params[b], bt.x0[b], float(bt.h[b]), int(bt.N[b]))
            window = R.spread(R.runs(wl, tol, max_iter, guard_B))[0]
            assert abs(int(iters[b]) - o["iters"]) <= window, (b, iters[b], o["iters"], window)
            seq = O.sequential(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b])
            assert relerr(g, seq) <= TOL_REL
        else:
            assert iters[b] == o["iters"] == max_iter
            seq = O.sequential(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b])
            k = int(iters[b])
            assert relerr(g[:k], seq[:k]) <= TOL_REL


def test_plain_vdp_batch_exact(pk):
    rng = np.random.default_rng(5)
    B = 24
    bt = W.Batch("vdp", W.VDP, rng.uniform(0.5, 2.0, (B, 1)), rng.uniform(-2, 2, (B, 2)),
                 np.full(B, 1e-3), rng.integers(1, 3000, B).astype(np.int64))
    bt.N[:3] = [1, 2, 3]
    out = run_batch(pk, bt, 1e-10, 60, 0.0)
    compare(bt, out, 1e-10, 60, 0.0)


@pytest.mark.parametrize("tile_elems", [2, 32])
def test_lorenz_batch_guarded(pk, tile_elems):
    # tile_elems=2 makes one CTA span 512 steps, so IVPs cross many CTAs
    bt = W.lorenz_batch(B=40, seed=1, n_min=1, n_max=4000)
    out = run_batch(pk, bt, 1e-12, 120, 100.0, tile_elems=tile_elems)
    compare(bt, out, 1e-12, 120, 100.0)


def test_lorenz_batch_capped(pk):
    bt = W.lorenz_batch(B=12, seed=2, n_min=3000, n_max=9000)
    out = run_batch(pk, bt, 1e-10, 15, 100.0, tile_elems=4)
    compare(bt, out, 1e-10, 15, 100.0)


def test_frozen_ivps_do_not_change(pk):
    # a mix of affine (one update) and nonlinear IVPs: the affine ones stop
    # after one update and must keep their converged trajectories
    rng = np.random.default_rng(9)
    B = 16
    params = np.stack([rng.uniform(0.5, 2, B), rng.uniform(0.0, 0.2, B)], 1)
    bt = W.Batch("osc", W.LINEAR_OSC, params, rng.uniform(-2, 2, (B, 2)), np.full(B, 1e-3),
                 rng.integers(100, 5000, B).astype(np.int64))
    out = run_batch(pk, bt, 1e-10, 10, 0.0, tile_elems=4)
    compare(bt, out, 1e-10, 10, 0.0)
    assert (out[2] == 1).all()


def test_full_batch_shape_sampled(pk):
    """4096 Lorenz IVPs of lengths in [2^10, 2^13] (the converging companion of
    the batched workload), checked on a sample of IVPs against the oracle."""
    bt = W.lorenz_batch(B=4096, seed=0, n_min=1 << 10, n_max=1 << 13)
    out = run_batch(pk, bt, 1e-12, 100, 100.0)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.integers(0, bt.B, 12).tolist()) | {0, bt.B - 1})
    compare(bt, out, 1e-12, 100, 100.0, sample=sample)


def test_host_arrays(pk):
    from paper_2511_01465_gb300 import pitn as P
    bt = W.lorenz_batch(B=5, seed=3, n_min=50, n_max=400)
    M = int(bt.N.sum())
    traj = np.zeros((M, 3))
    offs = np.zeros(bt.B + 1, dtype=np.int64)
    iters = np.zeros(bt.B, dtype=np.int32)
    status = np.zeros(bt.B, dtype=np.int32)
    res = np.zeros(bt.B)
    rc = P.pitn_solve_batch(bt.system, bt.B, bt.params, bt.x0, bt.h, bt.N, 3, 1e-12, 60, traj, offs,
                            iters, status, res, P.make_options(guard_B=100.0))
    assert rc in (P.PITN_OK, P.PITN_NOT_CONVERGED)
    compare(bt, (traj, offs, iters, status, res), 1e-12, 60, 100.0)


def test_batch_argument_errors(pk):
    from paper_2511_01465_gb300 import pitn as P
    bt = W.lorenz_batch(B=3, seed=3, n_min=5, n_max=10)
    bt.N[1] = 0
    M = int(np.maximum(bt.N, 0).sum())
    z = np.zeros((M, 3))
    rc = P.pitn_solve_batch(bt.system, bt.B, bt.params, bt.x0, bt.h, bt.N, 3, 1e-10, 5, z,
                            np.zeros(4, dtype=np.int64), np.zeros(3, dtype=np.int32),
                            np.zeros(3, dtype=np.int32), None, None)
    assert rc == P.PITN_EINVAL


@pytest.mark.parametrize("block", [512, 256, 128, 64])
@pytest.mark.parametrize("kind", ["vdp_plain", "lorenz_guard"])
def test_per_ivp_path(pk, block, kind):
    """The per-IVP path (one CTA solves each IVP whole, taken longest first)
    pinned through the tuner's cache: the same parity bar as the segmented
    path, lengths from 1 step to many steps per thread."""
    from paper_2511_01465_gb300 import pitn as P
    if kind == "vdp_plain":
        # plain Newton on van der Pol stays rounding-robust up to ~3000 steps
        # (longer IVPs can diverge on one side of a rounding difference)
        rng = np.random.default_rng(5)
        B = 24
        bt = W.Batch("vdp", W.VDP, rng.uniform(0.5, 2.0, (B, 1)), rng.uniform(-2, 2, (B, 2)),
                     np.full(B, 1e-3), rng.integers(1, 3000, B).astype(np.int64))
        bt.N[:4] = [1, 2, 3, 257]
        tol, it, gb = 1e-10, 60, 0.0
    else:
        bt = W.lorenz_batch(B=40, seed=3, n_min=1, n_max=3000)
        tol, it, gb = 1e-10, 50, 100.0
    M = int(bt.N.sum())
    key = f"batch:{bt.system}:{bt.d}:{M.bit_length() - 1}:{1 if gb > 0 else 0}"
    P.pitn_tune_clear()
    P.pitn_tune_set(key, block, 0)
    try:
        out = run_batch(pk, bt, tol, it, gb)
    finally:
        P.pitn_tune_clear()
    compare(bt, out, tol, it, gb)


def test_default_shape_takes_per_ivp_path(pk):
    """Untuned, a batch whose longest IVP is at most one CTA's share of the
    steps runs on the per-IVP path (three launches: init, the persistent
    solve, finalize) and matches the oracle IVP by IVP."""
    from paper_2511_01465_gb300 import pitn as P
    rng = np.random.default_rng(21)
    B = 1500
    bt = W.Batch("vdp", W.VDP, rng.uniform(0.5, 2.0, (B, 1)), rng.uniform(-2, 2, (B, 2)),
                 np.full(B, 1e-3), rng.integers(40, 160, B).astype(np.int64))
    bt.N[:3] = [1, 2, 3]
    P.pitn_tune_clear()
    P.pitn_tune_enable(False)
    l0 = pk.pitn_launch_count()
    out = run_batch(pk, bt, 1e-10, 60, 0.0)
    assert pk.pitn_launch_count() - l0 == 3
    compare(bt, out, 1e-10, 60, 0.0)


# ---------------------------------------------------------------------------
# The reduced-precision scans on the per-IVP path (an inexact Newton step;
# residual, stopping test and update in FP64): every IVP the FP64 oracle
# solves is solved, its FP64 residual re-checked by the oracle, its iterate
# within the path's bar (FP32 scan 1e-6, float-float 1e-10) of the oracle's
# at the same count, else of the sequential root beyond the oracle's own
# distance from it; the float-float solve's plain-Newton counts equal the
# oracle's.
# ---------------------------------------------------------------------------
def reduced_case(kind):
    if kind == "vdp_plain":
        rng = np.random.default_rng(5)
        B = 24
        bt = W.Batch("vdp", W.VDP, rng.uniform(0.5, 2.0, (B, 1)), rng.uniform(-2, 2, (B, 2)),
                     np.full(B, 1e-3), rng.integers(1, 3000, B).astype(np.int64))
        bt.N[:4] = [1, 2, 3, 257]
        return bt, 60, 0.0
    if kind == "osc_plain":
        rng = np.random.default_rng(8)
        B = 16
        bt = W.Batch("osc", W.LINEAR_OSC, np.column_stack([rng.uniform(0.5, 2.0, B), rng.uniform(0.0, 0.3, B)]),
                     rng.uniform(-2, 2, (B, 2)), np.full(B, 1e-3), rng.integers(1, 5000, B).astype(np.int64))
        return bt, 10, 0.0
    return W.lorenz_batch(B=40, seed=3, n_min=1, n_max=3000), 400, 100.0


@pytest.mark.parametrize("precision", ["fp32", "ff"])
@pytest.mark.parametrize("kind", ["vdp_plain", "osc_plain", "lorenz_guard"])
def test_reduced_precision_batch(pk, precision, kind):
    from paper_2511_01465_gb300 import pitn as P
    prec = P.PITN_PREC_MIXED_FP32 if precision == "fp32" else P.PITN_PREC_FP64_FF
    bar = 1e-6 if precision == "fp32" else 1e-10
    tol = 1e-11
    bt, it, gb = reduced_case(kind)
    traj, offs, iters, status, res = run_batch(pk, bt, tol, it, gb, precision=prec)
    assert offs[0] == 0 and np.array_equal(np.diff(offs), bt.N)
    solved = 0
    for b in range(bt.B):
        o = O.newton(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b], tol, it, guard_B=gb)
        if o["status"] != O.OK:
            continue
        solved += 1
        g = traj[offs[b]:offs[b + 1]]
        assert status[b] == O.OK and res[b] <= tol, (b, status[b], res[b])
        _, r, nf = O.residual(bt.system, bt.params[b], bt.x0[b], bt.h[b], g)
        assert not nf and r <= tol * (1 + 1e-6), (b, r)
        if iters[b] == o["iters"]:
            assert relerr(g, o["traj"]) <= bar, (b, relerr(g, o["traj"]))
        else:
            # another count: the iterate stops elsewhere within the tolerance;
            # against the sequential root, allowing the FP64 iterate's own
            # distance from it at this tolerance
            seq = O.sequential(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b])
            assert relerr(g, seq) <= bar + relerr(o["traj"], seq), (b, relerr(g, seq))
        if precision == "ff" and gb <= 0:
            assert iters[b] == o["iters"], (b, iters[b], o["iters"])
    assert solved >= bt.B // 2


def test_reduced_precision_batch_paths(pk):
    """The reduced-precision scans exist on the per-IVP path only: a tiled
    (segmented) request is an argument error, a pinned segmented shape is
    unsupported, a pinned per-IVP shape runs."""
    from paper_2511_01465_gb300 import pitn as P
    bt = W.lorenz_batch(B=8, seed=1, n_min=10, n_max=200)
    with pytest.raises(P.PitnError):
        run_batch(pk, bt, 1e-10, 50, 100.0, tile_elems=16, precision=P.PITN_PREC_MIXED_FP32)
    M = int(bt.N.sum())
    key = f"batch:{bt.system}:{bt.d}:{M.bit_length() - 1}:1:f32"
    P.pitn_tune_clear()
    try:
        P.pitn_tune_set(key, 256, 16)
        with pytest.raises(P.PitnError):
            run_batch(pk, bt, 1e-10, 50, 100.0, precision=P.PITN_PREC_MIXED_FP32)
        P.pitn_tune_set(key, 64, 0)
        out = run_batch(pk, bt, 1e-10, 50, 100.0, precision=P.PITN_PREC_MIXED_FP32)
        assert (out[3] == O.OK).all()
    finally:
        P.pitn_tune_clear()


@pytest.mark.parametrize("tile_elems", [0, 16])
def test_batch_work_counts(pk, tile_elems):
    """pitn_batch_work: the kernels' own counts of the steps they evaluated
    and replayed.  At most every step of an IVP in each of its passes
    (residual passes = updates + 1, replays = updates), fewer when the guard
    leaves a fill region, and at least one evaluation per pass."""
    from paper_2511_01465_gb300 import pitn as P
    bt = W.lorenz_batch(B=40, seed=3, n_min=1, n_max=3000)
    out = run_batch(pk, bt, 1e-10, 50, 100.0, tile_elems=tile_elems)
    iters = out[2].astype(np.int64)
    ev, rep = P.pitn_batch_work()
    assert 0 < ev <= int((bt.N * (iters + 1)).sum())
    assert 0 <= rep <= int((bt.N * iters).sum())
    assert ev >= int((iters + 1).sum())
