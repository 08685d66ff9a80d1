"""GPU parity of the adjoint (pitn_backward) against the oracle's sequential
reverse recursion, central finite differences (eps = 1e-6) and autograd."""
import numpy as np
import pytest

import oracle as O
from paper_2511_01465_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01465_gb300 as pk
    return pk


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def sequential_batch(bt):
    return np.concatenate([O.sequential(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b])
                           for b in range(bt.B)])


@pytest.mark.parametrize("kind", ["vdp", "lorenz", "osc"])
@pytest.mark.parametrize("ckpt", [256, 1024, 2048])
def test_backward_against_oracle_adjoint(pk, kind, ckpt):
    rng = np.random.default_rng(4)
    B = 7
    N = rng.integers(1, 3000, B).astype(np.int64)
    N[:2] = [1, 2]
    if kind == "vdp":
        bt = W.Batch("v", W.VDP, rng.uniform(0.5, 2, (B, 1)), rng.uniform(-2, 2, (B, 2)), np.full(B, 1e-3), N)
    elif kind == "lorenz":
        bt = W.Batch("l", W.LORENZ63, np.stack([rng.uniform(8, 12, B), rng.uniform(20, 35, B),
                                                rng.uniform(2, 3, B)], 1),
                     rng.normal(0, 5, (B, 3)), np.full(B, 1e-3), N)
    else:
        bt = W.Batch("o", W.LINEAR_OSC, np.stack([rng.uniform(0.5, 2, B), rng.uniform(0, 0.2, B)], 1),
                     rng.uniform(-2, 2, (B, 2)), np.full(B, 1e-3), N)
    traj = sequential_batch(bt)
    gt = rng.normal(0, 1, traj.shape)
    gN = rng.normal(0, 1, (B, bt.d))
    dev = "cuda"
    gx0, gp = pk.backward(bt.system, bt.params, bt.x0, bt.h, bt.N, torch.tensor(traj, device=dev),
                          grad_traj=torch.tensor(gt, device=dev), grad_xN=torch.tensor(gN, device=dev),
                          ckpt_every=ckpt)
    gx0, gp = gx0.cpu().numpy(), gp.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(bt.N)])
    for b in range(B):
        s, e = offs[b], offs[b + 1]
        ox, op = O.adjoint(bt.system, bt.params[b], bt.x0[b], bt.h[b], traj[s:e], grad_traj=gt[s:e],
                           grad_xN=gN[b])
        assert rel(gx0[b], ox) <= 1e-10, (b, gx0[b], ox)
        assert rel(gp[b], op) <= 1e-10, (b, gp[b], op)


def test_differentiation_workload_vs_fd(pk):
    """256 Van der Pol IVPs, N = 2^14, h = 1e-3, loss sum_i ||x_N^i - (1,0)||^2:
    forward by the batched Newton solve, gradients by the adjoint scan with
    checkpoints every 1024 steps; checked against the oracle adjoint on every
    IVP and central differences (eps = 1e-6) on a sample."""
    bt = W.vdp_adjoint_batch()
    dev = "cuda"
    traj, offs, iters, status, res = pk.solve_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, 1e-12, 200,
                                                    guard_B=100.0)
    assert (status.cpu().numpy() == 0).all()
    offs = offs.cpu().numpy()
    last = torch.tensor(offs[1:] - 1, device=dev)
    target = torch.tensor([1.0, 0.0], dtype=torch.float64, device=dev)
    gN = 2.0 * (traj[last] - target)
    gx0, gp = pk.backward(bt.system, bt.params, bt.x0, bt.h, bt.N, traj, grad_xN=gN.contiguous(),
                          ckpt_every=1024)
    gx0, gp, tr = gx0.cpu().numpy(), gp.cpu().numpy(), traj.cpu().numpy()
    for b in range(bt.B):
        s, e = offs[b], offs[b + 1]
        ox, op = O.adjoint(bt.system, bt.params[b], bt.x0[b], bt.h[b], tr[s:e],
                           grad_xN=2.0 * (tr[e - 1] - [1.0, 0.0]))
        assert rel(gx0[b], ox) <= 1e-10 and rel(gp[b], op) <= 1e-10, b
    eps = 1e-6
    for b in (0, 17, 101, 255):
        def loss(mu, x0):
            t = O.sequential(bt.system, [mu], x0, bt.h[b], bt.N[b])
            return float(((t[-1] - [1.0, 0.0]) ** 2).sum())
        mu, x0 = bt.params[b, 0], bt.x0[b]
        fd_mu = (loss(mu + eps, x0) - loss(mu - eps, x0)) / (2 * eps)
        fd_x = [(loss(mu, x0 + e) - loss(mu, x0 - e)) / (2 * eps) for e in np.eye(2) * eps]
        scale = max(1.0, abs(fd_mu), np.abs(fd_x).max())
        assert abs(gp[b, 0] - fd_mu) <= 1e-5 * scale, (b, gp[b, 0], fd_mu)
        assert np.abs(gx0[b] - fd_x).max() <= 1e-5 * scale, (b, gx0[b], fd_x)


@pytest.mark.parametrize("precision", [0, 2, 3], ids=["fp64", "fp32_scan", "float_float_scan"])
def test_autograd_function(pk, precision):
    from paper_2511_01465_gb300.autograd import odesolve
    bt = W.vdp_adjoint_batch(B=8, N=3000)
    dev = "cuda"
    params = torch.tensor(bt.params, device=dev, requires_grad=True)
    x0 = torch.tensor(bt.x0, device=dev, requires_grad=True)
    traj, offs, status = odesolve(bt.system, params, x0, torch.tensor(bt.h), torch.tensor(bt.N),
                                  tol=1e-12, max_iter=100, precision=precision)
    assert (status.cpu().numpy() == 0).all()
    last = offs[1:] - 1
    loss = ((traj[last] - torch.tensor([1.0, 0.0], dtype=torch.float64, device=dev)) ** 2).sum()
    loss.backward()
    tr = traj.detach().cpu().numpy()
    o = offs.cpu().numpy()
    for b in range(bt.B):
        s, e = o[b], o[b + 1]
        ox, op = O.adjoint(bt.system, bt.params[b], bt.x0[b], bt.h[b], tr[s:e],
                           grad_xN=2.0 * (tr[e - 1] - [1.0, 0.0]))
        assert rel(x0.grad[b].cpu().numpy(), ox) <= 1e-10
        assert rel(params.grad[b].cpu().numpy(), op) <= 1e-10


@pytest.mark.parametrize("precision,bar", [(3, 1e-10), (2, 1e-6)], ids=["float_float", "fp32"])
def test_gradients_through_reduced_precision_forward(pk, precision, bar):
    """The differentiation workload with its forward batch solved by the
    float-float or the FP32 scan (the adjoint itself FP64) at tol 1e-12: every
    IVP converges, and the gradients match the oracle adjoint on the returned
    trajectories to 1e-10 (the adjoint is exact on any trajectory) and the
    FP64-forward gradients to the scan's bar."""
    bt = W.vdp_adjoint_batch()
    dev = "cuda"
    grads = []
    for prec in (0, precision):
        traj, offs, iters, status, res = pk.solve_batch(bt.system, bt.params, bt.x0, bt.h, bt.N, 1e-12, 200,
                                                        guard_B=100.0, precision=prec)
        assert (status.cpu().numpy() == 0).all()
        last = offs[1:] - 1
        target = torch.tensor([1.0, 0.0], dtype=torch.float64, device=dev)
        gN = (2.0 * (traj[last] - target)).contiguous()
        gx0, gp = pk.backward(bt.system, bt.params, bt.x0, bt.h, bt.N, traj, grad_xN=gN, ckpt_every=1024)
        grads.append((gx0.cpu().numpy(), gp.cpu().numpy(), traj.cpu().numpy(), offs.cpu().numpy()))
    (gx_ref, gp_ref, _, _), (gx, gp, tr, offs) = grads
    for b in (0, 17, 101, 255):
        s, e = offs[b], offs[b + 1]
        ox, op = O.adjoint(bt.system, bt.params[b], bt.x0[b], bt.h[b], tr[s:e],
                           grad_xN=2.0 * (tr[e - 1] - [1.0, 0.0]))
        assert rel(gx[b], ox) <= 1e-10 and rel(gp[b], op) <= 1e-10, b
    assert np.abs(gp - gp_ref).max() <= bar * np.abs(gp_ref).max()
    assert np.abs(gx - gx_ref).max() <= bar * np.abs(gx_ref).max()
