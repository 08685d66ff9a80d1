"""A CPU shard backend for the time-sharded driver, for tests of its exchange
logic without a GPU (test infrastructure: it calls the oracle's step map).

It has the interface of paper_2511_01465_gb300.timeshard.CudaShard and the
semantics of the library's pitn_shard_* calls, written plainly: the
residual of eq. 3.8 from the state before the shard, the elements of eq. 3.4
composed in order by eq. 3.3 into the shard aggregate, and the sequential
replay of eq. 3.13 from the incoming correction, with the guard's lazy fill.
"""
from __future__ import annotations

import numpy as np

import oracle as O

MASK = 0x7FFFFFFFFFFFFFFF


def abs_bits(v):
    """The bit pattern of |v| as an int64 (NaN orders above +inf)."""
    return int(np.array([v], dtype=np.float64).view(np.int64)[0]) & MASK


class NumpyShard:
    def __init__(self, system, params, h, n, d, guard_B, device="cpu"):
        self.sys, self.p, self.h, self.n, self.d = system, np.asarray(params, dtype=np.float64), h, n, d
        self.cap = guard_B if (guard_B > 0 and np.isfinite(guard_B)) else np.finfo(np.float64).max
        self.elems = None

    def _states(self, X, x_prev, q):
        X = np.asarray(X.cpu() if hasattr(X, "cpu") else X, dtype=np.float64)
        xp = np.asarray(x_prev.cpu() if hasattr(x_prev, "cpu") else x_prev, dtype=np.float64)
        xs = X.copy()
        if q < self.n:
            xs[q:] = X[q - 1] if q > 0 else xp
        return xs, xp

    def pass_(self, x_prev, holds_first, X, q_local):
        import torch
        xs, xp = self._states(X, x_prev, q_local)
        d = self.d
        P, c = np.eye(d), np.zeros(d)
        elems, m = [], 0
        prev = xp
        for k in range(self.n):
            phi, J, _ = O.step(self.sys, self.p, self.h, prev, jac=True)
            r = xs[k] - phi
            for v in r:
                m = max(m, abs_bits(v))
            F = np.zeros((d, d)) if (holds_first and k == 0) else J
            elems.append((F, r))
            P, c = F @ P, F @ c - r
            prev = xs[k]
        self.elems, self.xs = elems, xs
        agg = np.concatenate([P.ravel(), c])
        return torch.tensor(agg, dtype=torch.float64), torch.tensor([m], dtype=torch.int64)

    def carry(self, r, aggs):
        import torch
        A = np.asarray(aggs.cpu(), dtype=np.float64)
        d = self.d
        z = np.zeros(d)
        for i in range(r):
            z = A[i, : d * d].reshape(d, d) @ z + A[i, d * d:]
        return torch.tensor(z, dtype=torch.float64)

    def update(self, z_in, Xn):
        import torch
        z = np.asarray(z_in.cpu(), dtype=np.float64)
        out = Xn.numpy()
        cut = self.n
        for k, (F, r) in enumerate(self.elems):
            z = F @ z - r
            out[k] = self.xs[k] + z
            if not (np.abs(z) <= self.cap).all():
                cut = k
                break
        return torch.tensor([cut], dtype=torch.int64)

    def finalize(self, X, x_prev, q_local, out):
        xs, _ = self._states(X, x_prev, q_local)
        out.numpy()[:] = xs

    def close(self):
        self.elems = None
