"""Host logic of the time-sharded solve (paper_2511_01465_gb300/timeshard.py)
on the CPU: the driver's exchange (halo and fill state, residual and cut
reductions, aggregate gather and carry order) with a plain CPU shard backend
(tests/timeshard_ref.py), as shards emulated by threads and as gloo ranks
(world size 2), against the oracle's unsharded Newton solve."""
import os
import socket
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle as O  # noqa: E402
from paper_2511_01465_gb300 import timeshard as T  # noqa: E402
from paper_2511_01465_gb300 import workloads as W  # noqa: E402
from timeshard_ref import NumpyShard  # noqa: E402

CASES = [
    # (name, workload, tol, max_iter, guard_B): rounding-robust problems
    ("vdp_plain", W.vdp(N=3001, h=1e-3), 1e-10, 60, 0.0),
    ("lorenz_guarded", W.lorenz(N=2000), 1e-10, 80, 100.0),
    ("lorenz_plain_diverges", W.lorenz(N=2000), 1e-10, 80, 0.0),
    ("osc_affine", W.damped_oscillator(N=997, h=1e-3), 1e-10, 5, 0.0),
]


def test_shard_bounds_partition():
    for N in (1, 2, 7, 1000, 1001):
        for R in range(1, min(N, 6) + 1):
            b = [T.shard_bounds(N, R, r) for r in range(R)]
            assert b[0][0] == 0 and b[-1][1] == N
            assert all(b[i][1] == b[i + 1][0] for i in range(R - 1))
            sizes = [e - s for s, e in b]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def run_threads(wl, tol, max_iter, guard_B, R):
    comms = T.ThreadComm.group(R)
    out = [None] * R
    errs = []

    def go(r):
        try:
            out[r] = T.solve_sharded(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, max_iter, comms[r],
                                     guard_B=guard_B, device="cpu", backend=NumpyShard)
        except BaseException as ex:  # noqa: BLE001
            errs.append(ex)
            comms[r].sh.barrier.abort()

    th = [threading.Thread(target=go, args=(r,)) for r in range(R)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return np.concatenate([o[0].numpy() for o in out]), [o[1] for o in out]


def check(o, traj, infos, N):
    for info in infos:   # every shard took the same decisions
        assert (info["iters"], info["status"], info["guard_index"]) == \
            (o["iters"], o["status"], o["guard_index"])
        assert np.array_equal(info["cut_history"], o["cuts"])
        np.testing.assert_allclose(info["res_history"], o["res_hist"], rtol=1e-9, atol=1e-15)
    assert traj.shape == o["traj"].shape
    assert np.abs(traj - o["traj"]).max() <= 1e-12 * np.abs(o["traj"]).max()


@pytest.mark.parametrize("R", [1, 2, 3, 5])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sharded_driver_matches_oracle_threads(case, R):
    _, wl, tol, it, B = case
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, it, guard_B=B)
    traj, infos = run_threads(wl, tol, it, B, R)
    check(o, traj, infos, wl.N)


def test_guard_fill_crosses_shards():
    """A guarded Lorenz solve capped early: the cut lies inside one shard and
    the shards after it hold only the fill state."""
    wl = W.lorenz(N=3000)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 3, guard_B=100.0)
    assert o["guard_index"] < wl.N // 2
    traj, infos = run_threads(wl, 1e-10, 3, 100.0, 4)
    check(o, traj, infos, wl.N)
    q = o["guard_index"]
    assert np.array_equal(traj[q:], np.broadcast_to(traj[q - 1], traj[q:].shape))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, name, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = {c[0]: c for c in CASES}[name]
        _, wl, tol, it, B = case
        traj, info = T.solve_sharded(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, it, T.TorchComm(),
                                     guard_B=B, device="cpu", backend=NumpyShard)
        parts = [None] * world
        dist.all_gather_object(parts, (traj.numpy(), info))
        if rank == 0:
            q.put(parts)
    except BaseException as ex:  # noqa: BLE001 -- reported to the test, which fails at once
        q.put(repr(ex))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["vdp_plain", "lorenz_guarded"])
def test_sharded_driver_gloo_world2(name):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=240)
    assert not isinstance(parts, str), parts
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, wl, tol, it, B = {c[0]: c for c in CASES}[name]
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, it, guard_B=B)
    check(o, np.concatenate([p[0] for p in parts]), [p[1] for p in parts], wl.N)
