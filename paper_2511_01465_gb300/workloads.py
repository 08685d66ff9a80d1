"""Seeded synthetic inputs for the solver's workloads.

This module holds input recipes only (parameters, initial values, lengths);
it contains none of the solver's arithmetic and imports nothing else from the
package, so the CUDA path, the tests and the CPU oracle can all draw the same
inputs from it.

Workloads (explicit Euler unless stated, FP64):
  * Lorenz-63, sigma=10, rho=28, beta=8/3, x0=(1,1,1), h=1e-3, N=8192;
  * Van der Pol, mu=1, x0=(2,0), h=1e-4, N=2^22;
  * damped linear oscillator x''+2 zeta omega x'+omega^2 x=0, omega=1,
    zeta=0.05, x0=(2,0), h=1e-4, N=2^22 (affine: one Newton update);
  * Fisher-KPP method of lines, 128 interior nodes on [0,1], D=1e-3,
    u0(x)=0.5(1+sin 2 pi x) exp(-20 (x-0.5)^2), h=5e-5, N=2^15;
  * batched Lorenz-63: B IVPs from numpy default_rng(seed), drawn as whole
    arrays in the order sigma~U[8,12], rho~U[20,35], beta~U[2,3],
    x0~N(0, 5^2 I) (B x 3), N_i~integers in [n_min, n_max] inclusive;
  * adjoint Van der Pol batch: default_rng(seed), mu~U[0.5,2] (B),
    x0~U[-2,2]^2 (B x 2), h=1e-3, N=2^14;
  * RK4 (Sec. 4.1): Van der Pol mu=1, x0=(0,1) on [0, 10], N = t_end / h,
    Newton guess = ones (the paper's);
  * backward Euler (Sec. 4.2): Dahlquist lambda=-1, y0=1 on [0, 4];
    Robertson k=(0.04, 3e7, 1e4), y0=(1,0,0) on [0, 500]; N = t_end / h,
    Newton guess = zeros (the paper's).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# system identifiers shared by the C ABI and the binding
LORENZ63, VDP, LINEAR_OSC, FKPP = 1, 2, 3, 4
DAHLQUIST, ROBERTSON = 6, 7


@dataclass
class Single:
    name: str
    system: int
    params: np.ndarray
    x0: np.ndarray
    h: float
    N: int

    @property
    def d(self) -> int:
        return int(self.x0.size)


@dataclass
class Batch:
    name: str
    system: int
    params: np.ndarray   # [B][P]
    x0: np.ndarray       # [B][d]
    h: np.ndarray        # [B]
    N: np.ndarray        # [B] int64

    @property
    def B(self) -> int:
        return int(self.N.size)

    @property
    def d(self) -> int:
        return int(self.x0.shape[1])


def lorenz(N: int = 8192, h: float = 1e-3) -> Single:
    return Single("lorenz63", LORENZ63, np.array([10.0, 28.0, 8.0 / 3.0]),
                  np.array([1.0, 1.0, 1.0]), h, N)


def vdp(N: int = 1 << 22, h: float = 1e-4, mu: float = 1.0) -> Single:
    return Single("van_der_pol", VDP, np.array([mu]), np.array([2.0, 0.0]), h, N)


def vdp_paper(h: float = 1e-5, t_end: float = 10.0, mu: float = 1.0) -> Single:
    return Single("van_der_pol_rk4", VDP, np.array([mu]), np.array([0.0, 1.0]), h, int(round(t_end / h)))


def damped_oscillator(N: int = 1 << 22, h: float = 1e-4) -> Single:
    return Single("damped_oscillator", LINEAR_OSC, np.array([1.0, 0.05]), np.array([2.0, 0.0]), h, N)


def fkpp_u0(d: int = 128) -> np.ndarray:
    xs = np.arange(1, d + 1, dtype=np.float64) / (d + 1)
    return 0.5 * (1.0 + np.sin(2.0 * math.pi * xs)) * np.exp(-20.0 * (xs - 0.5) ** 2)


def fkpp(d: int = 128, N: int = 1 << 15, h: float = 5e-5, D: float = 1e-3) -> Single:
    return Single("fisher_kpp", FKPP, np.array([D]), fkpp_u0(d), h, N)


def lorenz_batch(B: int = 4096, seed: int = 0, n_min: int = 1 << 10, n_max: int = 1 << 16,
                 h: float = 1e-3) -> Batch:
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(8.0, 12.0, B)
    rho = rng.uniform(20.0, 35.0, B)
    beta = rng.uniform(2.0, 3.0, B)
    x0 = rng.normal(0.0, 5.0, (B, 3))
    N = rng.integers(n_min, n_max, B, endpoint=True).astype(np.int64)
    params = np.stack([sigma, rho, beta], axis=1)
    return Batch("lorenz63_batch", LORENZ63, np.ascontiguousarray(params), np.ascontiguousarray(x0),
                 np.full(B, h), N)


def vdp_adjoint_batch(B: int = 256, seed: int = 0, N: int = 1 << 14, h: float = 1e-3) -> Batch:
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.5, 2.0, B)
    x0 = rng.uniform(-2.0, 2.0, (B, 2))
    return Batch("van_der_pol_adjoint", VDP, np.ascontiguousarray(mu[:, None]), np.ascontiguousarray(x0),
                 np.full(B, h), np.full(B, N, dtype=np.int64))


def dahlquist(h: float = 1e-1, lam: float = -1.0, t_end: float = 4.0) -> Single:
    return Single("dahlquist", DAHLQUIST, np.array([lam]), np.array([1.0]), h, int(round(t_end / h)))


def robertson(h: float = 1e-1, t_end: float = 500.0) -> Single:
    return Single("robertson", ROBERTSON, np.array([0.04, 3e7, 1e4]), np.array([1.0, 0.0, 0.0]), h,
                  int(round(t_end / h)))
