"""Rounding spread of guarded Newton solves, measured on the oracle.

With the divergence guard (reading R8, not in the paper) every Newton step
cuts the trajectory at the first correction that exceeds the bound B.
Beyond the converged prefix the corrections grow exponentially, so where the
cut falls depends on how the step was rounded, and with it the number of
Newton updates a guarded solve takes.  Rounding alone is measured here: the
oracle (oracle/pitn_oracle.c) is built in rounding variants of the same
mathematics -- FMA contraction, reversed summation order, a regrouped
residual, blocked bracketings of the recursion of eq. 3.13 (exact in real
arithmetic by the associativity of Lemma 3.1) and all of these at once --
and every variant solves the same problem.  What they agree on is fixed by
the mathematics and FP64 rounding; what they spread over is not.

The GPU parity bar for a guarded solve is then:
  - the status equals the oracle's;
  - the Newton count is within the variants' spread of the oracle's,
    window = max over variants of |iters_variant - iters_oracle|
    (0: the count must be equal);
  - the cut of every Newton step before the first step at which any variant
    cut elsewhere than the oracle is equal to the oracle's;
  - the residual history equals the oracle's (relative 1e-6) up to the first
    evaluation at which any variant's differs by more than that: the
    residual of a guarded iterate is largest next to the cut, where the
    corrections have grown exponentially, so it carries amplified rounding
    even while every variant cuts at the same step.
A scan in reduced precision rounds the Newton step more coarsely than any
FP64 order.  For the float-float scan (pairs of 24-bit floats, 48 significant
bits) the spread also takes the oracle's 48-bit-scan variant (s48: the
recursion's Jacobian entries, residuals and corrections rounded to 48 bits),
which models that precision with the same mathematics.
Only the oracle's code runs here.
"""
from __future__ import annotations

import numpy as np

import oracle as O

VARIANTS = list(O.VARIANTS)


def runs(wl, tol, max_iter, guard_B, method=O.EULER, guess=None, scan48=False):
    """The oracle and each rounding variant on one problem: {None: ..., name: ...}
    (with scan48, the 48-bit-scan variant as well)."""
    out = {}
    for v in [None] + VARIANTS + (list(O.SCAN_VARIANTS) if scan48 else []):
        out[v] = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, max_iter, guard_B=guard_B,
                          guess=guess, method=method, variant=v)
    return out


def first_difference(a, b):
    """First index at which two cut sequences differ (the shorter length if none)."""
    m = min(len(a), len(b))
    for i in range(m):
        if int(a[i]) != int(b[i]):
            return i
    return m


RES_RTOL, RES_ATOL = 1e-6, 1e-13


def first_res_difference(a, b):
    """First residual evaluation at which two histories differ by more than
    RES_RTOL relative (RES_ATOL absolute), the shorter length if none."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    m = min(len(a), len(b))
    bad = np.abs(a[:m] - b[:m]) > RES_RTOL * np.abs(b[:m]) + RES_ATOL
    return int(np.argmax(bad)) if bad.any() else m


def spread(rs):
    """(window, first_div, first_res_div) of a runs() result: the largest
    count difference of a variant from the oracle, the first Newton step at
    which a variant's cut differs from the oracle's, and the first residual
    evaluation at which a variant's residual differs from the oracle's."""
    ref = rs[None]
    window = max(abs(r["iters"] - ref["iters"]) for r in rs.values())
    first_div = min(first_difference(ref["cuts"], r["cuts"]) for r in rs.values())
    first_res_div = min(first_res_difference(r["res_hist"], ref["res_hist"]) for r in rs.values())
    return int(window), int(first_div), int(first_res_div)


def rejected_cut_window(rs):
    """For a plain solve that ends on a non-finite correction: the largest
    distance of a variant's index of that rejected correction from the
    oracle's (where a diverging correction leaves the FP64 range moves with
    rounding), or 0 when the solve does not end that way."""
    ref = rs[None]
    if len(ref["cuts"]) <= ref["iters"]:
        return 0
    return max(abs(int(r["cuts"][-1]) - int(ref["cuts"][-1])) for r in rs.values())


def check_guarded(gpu_status, gpu_iters, gpu_cuts, gpu_hist, ref, window, first_div, first_res_div):
    """Asserts the GPU outcome of a guarded solve against the oracle's `ref`
    (a dict with status, iters, cuts, res_hist) under the measured spread."""
    assert gpu_status == ref["status"], (gpu_status, ref["status"])
    assert abs(int(gpu_iters) - int(ref["iters"])) <= window, (gpu_iters, ref["iters"], window)
    k = min(first_div, len(ref["cuts"]))
    gc = np.asarray(gpu_cuts[:k], dtype=np.int64)
    rc = np.asarray(ref["cuts"][:k], dtype=np.int64)
    assert len(gc) == k and np.array_equal(gc, rc), (first_difference(gc, rc), k)
    h = min(first_res_div, first_div + 1, len(ref["res_hist"]), len(gpu_hist))
    np.testing.assert_allclose(np.asarray(gpu_hist[:h]), np.asarray(ref["res_hist"][:h]),
                               rtol=RES_RTOL, atol=RES_ATOL)
