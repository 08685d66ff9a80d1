"""Time-sharded Newton solve of one IVP over several GPUs (not in the paper,
which runs on one GPU).

Shard r of R owns the contiguous steps [s_r, s_r + n_r) of the trajectory
and one library plan (``pitn_shard_*``, include/pitn.h), which runs its
shard-local work on its device: the residual and element fold (eqs. 3.8,
3.4), the shard aggregate (eq. 3.3), the replay of eq. 3.13 and the guard
cut.  Per Newton iteration the shards exchange, through a communicator:

  1. the raw last state of every shard and the guard's fill state x_{q-1}
     (one all-gather of 2 d doubles per shard): shard r's halo is shard
     r-1's last state while the cut q lies at or after s_r, else the fill
     state (x0 when q = 0);
  2. the largest residual, reduced as its bit pattern (all-reduce max):
     every shard then takes the same decision (non-finite, tol, max_iter);
  3. the shard aggregates ((d^2 + d) doubles each, all-gather): shard r
     composes those of shards 0 .. r-1 into its incoming correction;
  4. the first guard cut, as a global step index (all-reduce min).

Communicators: ``TorchComm`` over a torch.distributed process group (NCCL on
GPUs, one rank per GPU); ``ThreadComm``, shards run as threads of one process
on one GPU, which exchange through host memory: no kernel waits on another
shard, every library call returns before the exchange.
"""
from __future__ import annotations

import threading

import numpy as np

from . import pitn as P

INF_BITS = 0x7FF0000000000000


def shard_bounds(N, R, r):
    """Steps [s, e) of shard r of R: contiguous, sizes differing by at most one."""
    base, extra = divmod(int(N), int(R))
    s = r * base + min(r, extra)
    return s, s + base + (1 if r < extra else 0)


def bits_to_double(b):
    return float(np.array([int(b)], dtype=np.int64).view(np.float64)[0])


class TorchComm:
    """Collectives of a torch.distributed process group on device tensors."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def all_gather(self, t):
        import torch
        shape = tuple(t.shape)
        flat = t.contiguous().reshape(-1)
        out = torch.empty(self.world * flat.numel(), dtype=t.dtype, device=t.device)
        self.dist.all_gather_into_tensor(out, flat, group=self.group)   # concatenated along dim 0
        return out.view((self.world,) + shape)

    def max_int(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return int(t.item())

    def min_int(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return int(t.item())


class ThreadComm:
    """R shards as threads of one process: collectives through host copies
    and a barrier.  comm = ThreadComm.group(R) gives one communicator per
    shard; run each shard's solve in its own thread."""

    class _Shared:
        def __init__(self, R):
            self.R = R
            self.slots = [None] * R
            self.barrier = threading.Barrier(R)

    def __init__(self, shared, rank):
        self.sh = shared
        self.rank = rank
        self.world = shared.R

    @staticmethod
    def group(R):
        sh = ThreadComm._Shared(R)
        return [ThreadComm(sh, r) for r in range(R)]

    def _exchange(self, value):
        self.sh.barrier.wait()
        self.sh.slots[self.rank] = value
        self.sh.barrier.wait()
        vals = list(self.sh.slots)
        self.sh.barrier.wait()
        return vals

    def all_gather(self, t):
        import torch
        vals = self._exchange(t.detach().cpu())
        return torch.stack(vals).to(t.device)

    def max_int(self, t):
        return max(int(v) for v in self._exchange(int(t.item())))

    def min_int(self, t):
        return min(int(v) for v in self._exchange(int(t.item())))


class CudaShard:
    """One shard's library plan on the current CUDA device."""

    def __init__(self, system, params, h, n, d, guard_B, device, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.d = d
        p = torch.as_tensor(np.asarray(params, dtype=np.float64), device=device)
        self.plan = P.shard_create(system, p, h, n, d, guard_B, stream)

    def pass_(self, x_prev, holds_first, X, q_local):
        t = self.torch
        agg = t.empty(self.d * self.d + self.d, dtype=t.float64, device=self.device)
        res = t.empty(1, dtype=t.int64, device=self.device)
        P.check(P.lib().pitn_shard_pass(self.plan, P._ptr(x_prev), int(holds_first), P._ptr(X), int(q_local),
                                        P._ptr(agg), P._ptr(res, np.int64)), "pitn_shard_pass")
        return agg, res

    def carry(self, r, aggs):
        t = self.torch
        z = t.empty(self.d, dtype=t.float64, device=self.device)
        P.check(P.lib().pitn_shard_carry(self.plan, int(r), P._ptr(aggs.contiguous()), P._ptr(z)),
                "pitn_shard_carry")
        return z

    def update(self, z_in, Xn):
        t = self.torch
        cut = t.empty(1, dtype=t.int64, device=self.device)
        P.check(P.lib().pitn_shard_update(self.plan, P._ptr(z_in), P._ptr(Xn), P._ptr(cut, np.int64)),
                "pitn_shard_update")
        return cut

    def finalize(self, X, x_prev, q_local, out):
        P.check(P.lib().pitn_shard_finalize(self.plan, P._ptr(X), P._ptr(x_prev), int(q_local), P._ptr(out)),
                "pitn_shard_finalize")

    def close(self):
        if self.plan is not None:
            P.lib().pitn_shard_destroy(self.plan)
            self.plan = None


def solve_sharded(system, params, x0, h, N, tol, max_iter, comm, *, guard_B=0.0, device="cuda",
                  backend=None):
    """The Newton solve of one IVP (explicit Euler, FP64) with shard
    comm.rank of comm.world.  Returns (local trajectory [n][d] of steps
    [s, e), info) with the same info on every shard: iters, status,
    final_res, guard_index, res_history, cut_history, bounds (s, e).

    backend: a factory (system, params, h, n, d, guard_B, device) -> shard
    object with pass_/carry/update/finalize/close (default CudaShard)."""
    import torch
    R, r = comm.world, comm.rank
    x0 = np.asarray(x0, dtype=np.float64)
    d = int(x0.size)
    N = int(N)
    if N < R:
        raise ValueError("every shard needs at least one step")
    s, e = shard_bounds(N, R, r)
    n = e - s
    make = backend or CudaShard
    sh = make(system, params, h, n, d, guard_B, device)
    guarded = guard_B > 0 and np.isfinite(guard_B)
    x0_t = torch.as_tensor(x0, device=device)
    X = x0_t.repeat(n, 1).contiguous()          # the constant guess x_k = x0
    Xn = torch.empty_like(X)
    zero = torch.zeros(d, dtype=torch.float64, device=device)
    q = N                                        # global lazy fill index
    hist, cuts = [], []
    it, status, final_res = 0, P.PITN_NOT_CONVERGED, 0.0

    def halo():
        """(x_prev, q_local): the state before this shard for the current iterate."""
        q_loc = min(max(q - s, 0), n)
        own = X[n - 1]
        fill = X[q - 1 - s] if s <= q - 1 < e else zero
        g = comm.all_gather(torch.stack([own, fill]))      # [R][2][d]
        if r == 0:
            xp = x0_t
        elif s <= q:
            xp = g[r - 1, 0]
        elif q == 0:
            xp = x0_t
        else:
            owner = next(i for i in range(R) if shard_bounds(N, R, i)[0] <= q - 1 < shard_bounds(N, R, i)[1])
            xp = g[owner, 1]
        return xp.contiguous(), q_loc

    try:
        while True:
            x_prev, q_loc = halo()
            agg, resb = sh.pass_(x_prev, r == 0, X, q_loc)
            rb = comm.max_int(resb)
            res = bits_to_double(rb)
            hist.append(res)
            final_res = res
            if rb >= INF_BITS:
                status = P.PITN_NONFINITE
                break
            if res <= tol:
                status = P.PITN_OK
                break
            if it == max_iter:
                status = P.PITN_NOT_CONVERGED
                break
            aggs = comm.all_gather(agg)                     # [R][d^2 + d]
            z = sh.carry(r, aggs)
            cut_l = sh.update(z, Xn)
            cl = int(cut_l.item())
            cut_g = torch.tensor([s + cl if cl < n else N], dtype=torch.int64, device=device)
            cut = comm.min_int(cut_g)
            cuts.append(cut)
            if not guarded and cut < N:
                status = P.PITN_NONFINITE
                break
            X, Xn = Xn, X
            q = cut if guarded else N
            it += 1
        x_prev, q_loc = halo()
        out = torch.empty_like(X)
        sh.finalize(X, x_prev, q_loc, out)
    finally:
        sh.close()
    # guard_index: the cut of the last accepted Newton step (a plain solve's
    # rejected last step is in cut_history only), as the single-GPU solve
    info = dict(iters=it, status=status, final_res=final_res, guard_index=cuts[it - 1] if it > 0 else N,
                res_history=np.array(hist), cut_history=np.array(cuts, dtype=np.int64), bounds=(s, e))
    return out, info


def solve_sharded_on_one_gpu(system, params, x0, h, N, tol, max_iter, R, *, guard_B=0.0, device="cuda"):
    """R shards of one solve as threads on one GPU (each its own plan and
    buffers, exchanging through host memory).  Returns the whole trajectory
    and the (shared) info."""
    import torch
    comms = ThreadComm.group(R)
    results = [None] * R
    errors = []

    def run(rk):
        try:
            results[rk] = solve_sharded(system, params, x0, h, N, tol, max_iter, comms[rk], guard_B=guard_B,
                                        device=device)
        except BaseException as ex:  # noqa: BLE001 -- re-raised below
            errors.append(ex)
            comms[rk].sh.barrier.abort()

    th = [threading.Thread(target=run, args=(rk,)) for rk in range(R)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errors:
        raise errors[0]
    traj = torch.cat([res[0] for res in results])
    return traj, results[0][1]
