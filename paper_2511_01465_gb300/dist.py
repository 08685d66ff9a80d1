"""Host-side multi-GPU logic: one process per GPU (torchrun).

The batched solve partitions into independent IVPs, so ranks shard the batch
and need no collective on the data path; only the benchmark's bookkeeping
(total steps solved, slowest rank's time) crosses ranks.  A single long IVP
does not shard here: ranks run independent replicas of it.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(N, world):
    """Contiguous IVP ranges [lo, hi) per rank with near-equal total steps."""
    N = np.asarray(N, dtype=np.int64)
    B = N.size
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.concatenate([[0], np.cumsum(N)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(cum, target, side="left"))
        if i > 0 and abs(cum[i - 1] - target) <= abs(cum[min(i, B)] - target):
            i -= 1  # the nearer IVP boundary
        bounds.append(min(max(i, bounds[-1]), B))
    bounds.append(B)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def shard_batch(bt, rank, world):
    """The rank's sub-batch (same Batch type, contiguous IVPs) and its IVP range."""
    lo, hi = shard_bounds(bt.N, world)[rank]
    sub = type(bt)(f"{bt.name}[{lo}:{hi}]", bt.system, bt.params[lo:hi], bt.x0[lo:hi], bt.h[lo:hi],
                   bt.N[lo:hi])
    return sub, (lo, hi)


def aggregate(steps_solved, ms, group=None):
    """(total steps over ranks, max time over ranks) with torch.distributed."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(steps_solved), float(ms)
    dev = "cpu" if dist.get_backend(group) == "gloo" else torch.device("cuda", torch.cuda.current_device())
    s = torch.tensor([float(steps_solved)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(s.item()), float(t.item())
