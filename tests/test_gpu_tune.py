"""The launch-shape autotuner: a tuned solve caches its shape and still
matches the oracle; the cache is cleared afterwards so later tests run with
the default shapes."""
import numpy as np
import pytest

import oracle as O
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    from paper_2511_01465_gb300 import pitn as P
    P.pitn_tune_clear()
    P.pitn_tune_enable(True)
    try:
        yield pk
    finally:
        P.pitn_tune_enable(False)
        P.pitn_tune_clear()


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max())


def test_tuned_single_solve(pk):
    from paper_2511_01465_gb300 import pitn as P
    wl = W.vdp(N=40000, h=1e-3)
    key = f"small:{wl.system}:2:{int(np.log2(wl.N))}:0"
    assert P.pitn_tune_get(key) is None
    traj, info = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
    shape = P.pitn_tune_get(key)
    assert shape is not None and shape[0] in (128, 256, 512) and 1 <= shape[1] <= 8
    # a short trajectory: the steps-per-thread floor is tuned too
    cmin = P.pitn_tune_get(key + ":c")
    assert cmin is not None and cmin[0] in (1, 2, 4)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
    assert (info["iters"], info["status"]) == (o["iters"], o["status"])
    assert relerr(traj.cpu().numpy(), o["traj"]) <= 1e-10
    # the cached shape is reused (no retuning): same bits on a second call
    traj2, info2 = pk.solve(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 60)
    assert torch.equal(traj, traj2)


def test_tuned_batch_solve(pk):
    from paper_2511_01465_gb300 import pitn as P
    rng = np.random.default_rng(6)
    B = 20
    bt = W.Batch("vdp", W.VDP, rng.uniform(0.5, 2.0, (B, 1)), rng.uniform(-2, 2, (B, 2)),
                 np.full(B, 1e-3), rng.integers(100, 4000, B).astype(np.int64))
    traj, offs, iters, status, res = pk.solve_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, 1e-10, 60)
    M = int(bt.N.sum())
    shape = P.pitn_tune_get(f"batch:{bt.system}:2:{int(np.log2(M))}:0")
    assert shape is not None and shape[0] in (128, 256) and shape[1] in (0, 8, 16, 32, 64)
    traj, offs = traj.cpu().numpy(), offs.cpu().numpy()
    for b in range(B):
        o = O.newton(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b], 1e-10, 60)
        assert int(iters[b]) == o["iters"] and int(status[b]) == o["status"]
        assert relerr(traj[offs[b]:offs[b + 1]], o["traj"]) <= 1e-10
