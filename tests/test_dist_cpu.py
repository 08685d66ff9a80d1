"""Multi-process host logic on CPU (gloo, world size 2): the batch shards
into contiguous IVP ranges that partition it, shard results reassemble into
the unsharded result, and the benchmark aggregation takes the sum of steps
and the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2511_01465_gb300 import dist as D  # noqa: E402
from paper_2511_01465_gb300 import workloads as W  # noqa: E402


def test_shard_bounds_partition():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        N = rng.integers(1, 1000, 37)
        b = D.shard_bounds(N, world)
        assert b[0][0] == 0 and b[-1][1] == 37
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        ideal = N.sum() / world
        for lo, hi in b:
            assert abs(N[lo:hi].sum() - ideal) <= N.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    bt = W.lorenz_batch(B=9, seed=4, n_min=20, n_max=300)
    sub, (lo, hi) = D.shard_batch(bt, rank, world)
    out = O.newton_batch(sub.system, sub.params, sub.x0, sub.h, sub.N, 1e-10, 60, guard_B=100.0) \
        if sub.B else None
    solved = int(sub.N[out["status"] == 0].sum()) if out else 0
    total, tmax = D.aggregate(solved, 10.0 * (rank + 1))
    gathered = [None] * world
    dist.all_gather_object(gathered, (lo, hi, out["iters"].tolist() if out else [],
                                      out["status"].tolist() if out else []))
    if rank == 0:
        q.put((total, tmax, gathered))
    dist.destroy_process_group()


def test_sharded_batch_matches_unsharded_gloo():
    import oracle as O
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    total, tmax, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    bt = W.lorenz_batch(B=9, seed=4, n_min=20, n_max=300)
    full = O.newton_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, 1e-10, 60, guard_B=100.0)
    iters, status = [], []
    for lo, hi, it, st in sorted(gathered):
        iters += it
        status += st
    assert iters == full["iters"].tolist() and status == full["status"].tolist()
    assert total == float(bt.N[full["status"] == 0].sum())
    assert tmax == 20.0
