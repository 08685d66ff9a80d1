"""The seeded synthetic inputs (paper_2511_01465_gb300/workloads.py) against
the recipes the bench configurations state: fixed systems with their stated
parameters, initial values, step sizes and lengths, and the seeded batches'
distributions (ranges, moments, reproducibility).  The generators hold no
arithmetic of the method."""
import math

import numpy as np
import pytest

from paper_2511_01465_gb300 import workloads as W


def test_fixed_configurations():
    lz = W.lorenz()
    assert (lz.system, lz.N, lz.h) == (W.LORENZ63, 8192, 1e-3)
    assert np.allclose(lz.params, [10.0, 28.0, 8.0 / 3.0]) and np.array_equal(lz.x0, [1.0, 1.0, 1.0])
    v = W.vdp()
    assert (v.system, v.N, v.h) == (W.VDP, 1 << 22, 1e-4)
    assert np.array_equal(v.params, [1.0]) and np.array_equal(v.x0, [2.0, 0.0])
    o = W.damped_oscillator()
    assert (o.system, o.N) == (W.LINEAR_OSC, 1 << 22) and np.array_equal(o.x0, [2.0, 0.0])
    r = W.vdp_paper()   # Sec. 4.1: x0 = (0, 1) on [0, 10]
    assert r.N == 1_000_000 and np.array_equal(r.x0, [0.0, 1.0]) and r.h * r.N == pytest.approx(10.0)
    rb = W.robertson(h=1e-4)   # Sec. 4.2: k = (0.04, 3e7, 1e4), y0 = (1, 0, 0) on [0, 500]
    assert rb.N == 5_000_000 and np.array_equal(rb.params, [0.04, 3e7, 1e4])
    assert np.array_equal(rb.x0, [1.0, 0.0, 0.0])


def test_fkpp_grid_and_initial_profile():
    f = W.fkpp()
    assert (f.system, f.d, f.N, f.h) == (W.FKPP, 128, 1 << 15, 5e-5) and np.array_equal(f.params, [1e-3])
    # interior nodes of [0, 1] with Dirichlet ends: u0 = 0.5 (1 + sin 2 pi x) exp(-20 (x - 0.5)^2)
    xs = np.arange(1, 129) / 129.0
    ref = 0.5 * (1.0 + np.sin(2.0 * math.pi * xs)) * np.exp(-20.0 * (xs - 0.5) ** 2)
    assert np.allclose(f.x0, ref, rtol=0, atol=1e-15)
    assert (f.x0 >= 0).all() and f.x0.max() <= 1.0


def test_lorenz_batch_distribution():
    bt = W.lorenz_batch()
    assert bt.B == 4096 and bt.d == 3 and (bt.h == 1e-3).all()
    s, r, b = bt.params.T
    assert 8 <= s.min() and s.max() <= 12 and 20 <= r.min() and r.max() <= 35 and 2 <= b.min() and b.max() <= 3
    assert abs(s.mean() - 10) < 0.1 and abs(r.mean() - 27.5) < 0.3 and abs(b.mean() - 2.5) < 0.03
    assert abs(bt.x0.mean()) < 0.2 and abs(bt.x0.std() - 5.0) < 0.1     # x0 ~ N(0, 25 I)
    assert bt.N.min() >= 1 << 10 and bt.N.max() <= 1 << 16 and bt.N.dtype == np.int64
    assert abs(bt.N.mean() - ((1 << 10) + (1 << 16)) / 2) < 1000       # uniform integer lengths
    again = W.lorenz_batch()
    assert np.array_equal(again.params, bt.params) and np.array_equal(again.N, bt.N)   # seeded
    other = W.lorenz_batch(seed=1)
    assert not np.array_equal(other.N, bt.N)


def test_adjoint_batch_distribution():
    bt = W.vdp_adjoint_batch()
    assert bt.B == 256 and bt.d == 2 and (bt.N == 1 << 14).all() and (bt.h == 1e-3).all()
    mu = bt.params[:, 0]
    assert 0.5 <= mu.min() and mu.max() <= 2.0 and abs(mu.mean() - 1.25) < 0.1
    assert -2 <= bt.x0.min() and bt.x0.max() <= 2 and abs(bt.x0.mean()) < 0.2
