"""Failure paths on the GPU, made on the host (no GPU fault, no hang).

Every in-kernel wait of the library is bounded: a grid barrier gives up
after a time limit, the tensor-core compose after a number of mbarrier
polls, and the call returns PITN_ETIMEOUT.  The tests shorten those limits
through pitn_debug_inject so that the waits run out at once, check the
status, and check that the device stays usable: the next solve with the
default limits matches the oracle.  A compose whose wait gave up waits for
the copies or the product already in flight before it frees its TMEM, so
the TMEM of the failed launch is free again for the next one.  An injected
failure of the scratch cache's allocation gives PITN_ENOMEM."""
import numpy as np
import pytest

import oracle as O
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_01465_gb300 import pitn
    yield pitn
    pitn.pitn_debug_inject(pitn.PITN_DEBUG_RESET)


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def small_solve(P, wl):
    dev = torch.device("cuda", 0)
    out = torch.empty((wl.N, wl.d), dtype=torch.float64, device=dev)
    rc, r = P.pitn_solve_ex(wl.system, wl.params, wl.x0, wl.h, wl.N, wl.d, 1e-10, 40, out, P.make_options())
    torch.cuda.synchronize()
    return rc, r, out.cpu().numpy()


def fkpp_solve(P, wl):
    dev = torch.device("cuda", 0)
    out = torch.empty((wl.N, wl.d), dtype=torch.float64, device=dev)
    rc, r = P.pitn_solve_ex(wl.system, wl.params, wl.x0, wl.h, wl.N, wl.d, 1e-10, 20, out,
                            P.make_options(precision=P.PITN_PREC_MIXED_BF16))
    torch.cuda.synchronize()
    return rc, r, out.cpu().numpy()


def test_grid_barrier_timeout_returns_etimeout(P):
    """A grid barrier that may wait only 1 ns gives up in the first CTA that
    arrives before the others: the solve returns PITN_ETIMEOUT; with the
    default limit the same solve then equals the oracle's."""
    wl = W.vdp(N=65536, h=1e-4)          # 64 CTAs: every pass has grid barriers
    assert P.pitn_debug_inject(P.PITN_DEBUG_GRID_WAIT_NS, 1) == P.PITN_OK
    try:
        rc, _, _ = small_solve(P, wl)
    finally:
        P.pitn_debug_inject(P.PITN_DEBUG_RESET)
    assert rc == P.PITN_ETIMEOUT
    rc, r, g = small_solve(P, wl)
    o = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, 1e-10, 40)
    assert rc == o["status"] == O.OK and r.iters == o["iters"]
    assert relerr(g, o["traj"]) <= 1e-10


@pytest.mark.parametrize("knob", ["load", "mma"])
def test_tensor_core_wait_timeout_returns_etimeout(P, knob):
    """The tensor-core compose of the mixed-precision Fisher-KPP scan with
    zero polls for its bulk copies, or for its product: PITN_ETIMEOUT, and the
    next solve (default limits, TMEM freed by the failed launch) is correct."""
    wl = W.fkpp(N=2000)
    what = P.PITN_DEBUG_LOAD_POLLS if knob == "load" else P.PITN_DEBUG_MMA_POLLS
    assert P.pitn_debug_inject(what, 0) == P.PITN_OK
    try:
        rc, _, _ = fkpp_solve(P, wl)
    finally:
        P.pitn_debug_inject(P.PITN_DEBUG_RESET)
    assert rc == P.PITN_ETIMEOUT
    rc, r, g = fkpp_solve(P, wl)
    seq = O.sequential(wl.system, wl.params, wl.x0, wl.h, wl.N)
    assert rc == P.PITN_OK and relerr(g, seq) <= 1e-6


def test_combine_primitive_timeout_then_correct(P):
    """pitn_affine_combine_delta with zero polls for the product returns
    PITN_ETIMEOUT; with the default limit it matches the oracle's combine
    (BF16 operands: the bounds of test_gpu_compose_tc.py)."""
    rng = np.random.default_rng(11)
    n = 3
    S2 = rng.uniform(-0.05, 0.05, (n, 128, 128)).astype(np.float32)
    S1 = rng.uniform(-0.05, 0.05, (n, 128, 128)).astype(np.float32)
    b2 = rng.normal(0, 1, (n, 128)).astype(np.float32)
    b1 = rng.normal(0, 1, (n, 128)).astype(np.float32)
    dev = torch.device("cuda", 0)
    # column-major storage: element (i, j) at [j][i]
    cm = lambda M: torch.tensor(np.ascontiguousarray(np.swapaxes(M, 1, 2)), device=dev)
    dS2, dS1 = cm(S2), cm(S1)
    db2, db1 = torch.tensor(b2, device=dev), torch.tensor(b1, device=dev)
    S = torch.empty_like(dS2)
    b = torch.empty_like(db2)
    assert P.pitn_debug_inject(P.PITN_DEBUG_MMA_POLLS, 0) == P.PITN_OK
    try:
        rc = P.pitn_affine_combine_delta(n, dS2, db2, dS1, db1, S, b)
    finally:
        P.pitn_debug_inject(P.PITN_DEBUG_RESET)
    assert rc == P.PITN_ETIMEOUT
    assert P.pitn_affine_combine_delta(n, dS2, db2, dS1, db1, S, b) == P.PITN_OK
    Sh = np.swapaxes(S.cpu().numpy(), 1, 2).astype(np.float64)
    bh = b.cpu().numpy().astype(np.float64)
    I = np.eye(128)
    for k in range(n):
        A, c = O.combine(I + S2[k].astype(np.float64), b2[k], I + S1[k].astype(np.float64), b1[k])
        assert np.abs((I + Sh[k]) - A).max() <= 128 * 0.05 * 0.05 * 2.0 ** -7
        assert np.abs(bh[k] - c).max() <= 128 * 0.05 * np.abs(b1[k]).max() * 2.0 ** -8


def test_allocation_failure_returns_enomem(P):
    """With the scratch cache emptied and its next growth refused, a solve
    returns PITN_ENOMEM and writes no trajectory; the next solve succeeds."""
    wl = W.lorenz(N=3000)
    assert P.pitn_release_workspace() == P.PITN_OK
    assert P.pitn_debug_inject(P.PITN_DEBUG_FAIL_ALLOCS, 1) == P.PITN_OK
    try:
        rc, _, _ = small_solve(P, wl)
    finally:
        P.pitn_debug_inject(P.PITN_DEBUG_RESET)
    assert rc == P.PITN_ENOMEM
    rc, r, g = small_solve(P, wl)
    assert rc in (P.PITN_OK, P.PITN_NOT_CONVERGED, P.PITN_NONFINITE)


def test_inject_rejects_unknown_settings(P):
    assert P.pitn_debug_inject(99, 0) == P.PITN_EINVAL
    assert P.pitn_debug_inject(P.PITN_DEBUG_FAIL_ALLOCS, -1) == P.PITN_EINVAL
