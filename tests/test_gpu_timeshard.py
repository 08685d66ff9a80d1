"""The time-sharded solve of one IVP (pitn_shard_* and timeshard.py) on one
GPU, its shards emulated as threads that exchange through host memory (no
kernel waits on another shard).  Against the oracle: plain solves bit-exact
in their integer outcomes, guarded ones within the measured rounding spread
(tests/rounding.py), trajectories within 1e-10."""
import json
import os

import numpy as np
import pytest

import oracle as O
import rounding as R
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_01465_gb300 import timeshard
    return timeshard


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("shards", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["vdp", "lorenz_plain", "osc"])
def test_sharded_plain_equals_oracle(T, kind, shards):
    wl = {"vdp": W.vdp(N=30001, h=1e-3), "lorenz_plain": W.lorenz(N=4099),
          "osc": W.damped_oscillator(N=65537, h=1e-3)}[kind]
    traj, info = T.solve_sharded_on_one_gpu(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60, shards)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
    assert (info["iters"], info["status"], info["guard_index"]) == (o["iters"], o["status"], o["guard_index"])
    # the accepted steps' cuts exactly; where plain Newton diverges, the index
    # at which the rejected correction overflows within the oracle's rounding
    # variants' spread of it (van der Pol, 30001 steps: 11026 and 11027,
    # stored by tests/golden/make_rounding_spread.py)
    k = o["iters"]
    assert len(info["cut_history"]) == len(o["cuts"])
    assert np.array_equal(info["cut_history"][:k], o["cuts"][:k])
    if len(o["cuts"]) > k:
        with open(os.path.join(HERE, "golden", "oracle_rounding_spread.json")) as f:
            win = json.load(f)["vdp_30001_h1e-3_plain_tol1e-10_it60"]["rejected_cut_window"] \
                if kind == "vdp" else 0
        assert abs(int(info["cut_history"][k]) - int(o["cuts"][k])) <= win
    np.testing.assert_allclose(info["res_history"], o["res_hist"], rtol=1e-6, atol=1e-13)
    assert relerr(traj.cpu().numpy(), o["traj"]) <= 1e-10


@pytest.mark.parametrize("shards", [2, 5])
def test_sharded_guarded_lorenz_8192(T, shards):
    """Guarded Lorenz-63, N = 8192, tol 1e-12: within the oracle's measured
    rounding spread, and the root to 1e-10."""
    with open(os.path.join(HERE, "golden", "oracle_rounding_spread.json")) as f:
        sp = json.load(f)["lorenz_8192_guard100_tol1e-12_it100"]
    ref = dict(sp["oracle"], res_hist=sp["oracle"]["res_history"])
    wl = W.lorenz()
    traj, info = T.solve_sharded_on_one_gpu(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-12, 100, shards,
                                            guard_B=100.0)
    R.check_guarded(info["status"], info["iters"], info["cut_history"], info["res_history"], ref, sp["window"],
                    sp["first_div"], sp["first_res_div"])
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    assert relerr(traj.cpu().numpy(), seq) <= 1e-10


def test_sharded_guard_cut_inside_a_shard(T):
    """Capped after 3 updates: the cut lies in the first shard, the shards
    after it read only the fill state; all integer outcomes equal."""
    wl = W.lorenz(N=3000)
    traj, info = T.solve_sharded_on_one_gpu(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 3, 4,
                                            guard_B=100.0)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 3, guard_B=100.0)
    assert (info["iters"], info["status"], info["guard_index"]) == (o["iters"], o["status"], o["guard_index"])
    assert np.array_equal(info["cut_history"], o["cuts"])
    g = traj.cpu().numpy()
    q = o["guard_index"]
    assert q < wl.N // 4
    assert relerr(g, o["traj"]) <= 1e-10
    assert np.array_equal(g[q:], np.broadcast_to(g[q - 1], g[q:].shape))


def test_shard_argument_errors(T):
    from paper_2511_01465_gb300 import pitn as P
    with pytest.raises(P.PitnError):
        P.shard_create(P.PITN_FKPP, np.ones(1), 1e-3, 10, 128)
    with pytest.raises(P.PitnError):
        P.shard_create(P.PITN_VDP, np.ones(1), 1e-3, 0, 2)
    plan = P.shard_create(P.PITN_VDP, np.ones(1), 1e-3, 10, 2)
    z = torch.zeros(2, dtype=torch.float64, device="cuda")
    Xn = torch.zeros((10, 2), dtype=torch.float64, device="cuda")
    cut = torch.zeros(1, dtype=torch.int64, device="cuda")
    # an update needs a pass first
    assert P.lib().pitn_shard_update(plan, P._ptr(z), P._ptr(Xn), P._ptr(cut, np.int64)) == P.PITN_EINVAL
    assert P.lib().pitn_shard_destroy(plan) == P.PITN_OK
