"""The dense delta-form combine of eq. 3.3 on the tensor cores (tcgen05,
BF16 operands, FP32 accumulation in TMEM), through the C ABI, against numpy
products of the same BF16-rounded operands and against the oracle's FP64
combine."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_01465_gb300 import pitn
    return pitn


def bf16(x):
    """float32 -> nearest-even bfloat16 -> float32 (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def run(P, S2, b2, S1, b1):
    n = S2.shape[0]
    dev = "cuda"
    # column-major storage: element (i, j) at [j][i]
    t = lambda M: torch.tensor(np.ascontiguousarray(np.swapaxes(M, 1, 2)), dtype=torch.float32, device=dev)
    v = lambda x: torch.tensor(x, dtype=torch.float32, device=dev)
    S = torch.empty((n, 128, 128), dtype=torch.float32, device=dev)
    b = torch.empty((n, 128), dtype=torch.float32, device=dev)
    rc = P.pitn_affine_combine_delta(n, t(S2), v(b2), t(S1), v(b1), S, b)
    assert rc == 0
    return np.swapaxes(S.cpu().numpy(), 1, 2).astype(np.float64), b.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("scale", [0.2, 3.0])
def test_combine_matches_bf16_products(P, scale):
    rng = np.random.default_rng(2)
    n = 6
    S2 = rng.uniform(-scale, scale, (n, 128, 128)).astype(np.float32)
    S1 = rng.uniform(-scale, scale, (n, 128, 128)).astype(np.float32)
    b2 = rng.normal(0, 1, (n, 128)).astype(np.float32)
    b1 = rng.normal(0, 1, (n, 128)).astype(np.float32)
    S, b = run(P, S2, b2, S1, b1)
    prod = np.einsum("nik,nkj->nij", bf16(S2).astype(np.float64), bf16(S1).astype(np.float64))
    ref = S2.astype(np.float64) + S1 + prod
    bound = 128 * scale * scale * 2.0 ** -22 + np.abs(ref) * 2.0 ** -22
    assert (np.abs(S - ref) <= bound).all(), np.abs(S - ref).max()
    # vector part: the same BF16 rows of S2 times the FP32 vector, FP32 accumulation
    bref = b2.astype(np.float64) + b1 + np.einsum("nik,nk->ni", bf16(S2).astype(np.float64), b1)
    assert np.abs(b - bref).max() <= 1e-5 * max(1.0, np.abs(bref).max())
    # operand order of eq. 3.3 (later element on the left) is the one computed
    wrong = S2.astype(np.float64) + S1 + np.einsum("nik,nkj->nij", S1.astype(np.float64), S2)
    assert np.abs(S - ref).max() < 1e-3 * np.abs(S - wrong).max()


def test_combine_agrees_with_oracle_combine(P):
    rng = np.random.default_rng(3)
    S2 = rng.uniform(-0.05, 0.05, (1, 128, 128)).astype(np.float32)
    S1 = rng.uniform(-0.05, 0.05, (1, 128, 128)).astype(np.float32)
    b2 = rng.normal(0, 1, (1, 128)).astype(np.float32)
    b1 = rng.normal(0, 1, (1, 128)).astype(np.float32)
    S, b = run(P, S2, b2, S1, b1)
    I = np.eye(128)
    A, bo = O.combine(I + S2[0].astype(np.float64), b2[0], I + S1[0].astype(np.float64), b1[0])
    # BF16 operands: the product term carries ~2^-8 relative error
    assert np.abs((I + S[0]) - A).max() <= 128 * 0.05 * 0.05 * 2.0 ** -7
    # the vector part carries the BF16 rounding of S2 (2^-9 relative per entry)
    assert np.abs(b[0] - bo).max() <= 128 * 0.05 * np.abs(b1).max() * 2.0 ** -8


def tf32_trunc(x):
    """float32 -> TF32 by dropping the low 13 mantissa bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def tf32_rn(x):
    """float32 -> TF32 rounded to nearest even (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0xFFF + ((u >> 13) & 1)) >> 13) << 13
    return u.astype(np.uint32).view(np.float32)


def run_tf32(P, S2, b2, S1, b1):
    n = S2.shape[0]
    dev = "cuda"
    t = lambda M: torch.tensor(np.ascontiguousarray(np.swapaxes(M, 1, 2)), dtype=torch.float32, device=dev)
    v = lambda x: torch.tensor(x, dtype=torch.float32, device=dev)
    S = torch.empty((n, 128, 128), dtype=torch.float32, device=dev)
    b = torch.empty((n, 128), dtype=torch.float32, device=dev)
    assert P.pitn_affine_combine_delta_tf32(n, t(S2), v(b2), t(S1), v(b1), S, b) == 0
    return np.swapaxes(S.cpu().numpy(), 1, 2).astype(np.float64), b.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("scale", [0.2, 3.0])
def test_tf32_combine_matches_products(P, scale):
    """TF32 operands: the product within the TF32 rounding of both operands
    (2^-10 relative each, whether truncated or rounded) of the exact one,
    and the operand order of eq. 3.3; the vector part in FP32."""
    rng = np.random.default_rng(7)
    n = 4
    S2 = rng.uniform(-scale, scale, (n, 128, 128)).astype(np.float32)
    S1 = rng.uniform(-scale, scale, (n, 128, 128)).astype(np.float32)
    b2 = rng.normal(0, 1, (n, 128)).astype(np.float32)
    b1 = rng.normal(0, 1, (n, 128)).astype(np.float32)
    S, b = run_tf32(P, S2, b2, S1, b1)
    exact = np.einsum("nik,nkj->nij", S2.astype(np.float64), S1.astype(np.float64))
    ref = S2.astype(np.float64) + S1 + exact
    bound = 128 * scale * scale * 2.0 ** -9 + np.abs(ref) * 2.0 ** -22
    assert (np.abs(S - ref) <= bound).all(), np.abs(S - ref).max()
    # the product of TF32 operands (truncated or rounded, whichever the tensor
    # core takes) to FP32 accumulation accuracy: BF16 operands would miss it
    # by ~2^-9 relative
    base = S2.astype(np.float64) + S1
    errs = []
    for cut in (tf32_trunc, tf32_rn):
        prod = np.einsum("nik,nkj->nij", cut(S2).astype(np.float64), cut(S1).astype(np.float64))
        errs.append(np.abs(S - (base + prod)).max())
    assert min(errs) <= 128 * scale * scale * 2.0 ** -18, errs
    bref = b2.astype(np.float64) + b1 + np.einsum("nik,nk->ni", S2.astype(np.float64), b1)
    assert np.abs(b - bref).max() <= 1e-5 * max(1.0, np.abs(bref).max())
    wrong = S2.astype(np.float64) + S1 + np.einsum("nik,nkj->nij", S1.astype(np.float64), S2)
    assert np.abs(S - ref).max() < 1e-3 * np.abs(S - wrong).max()
