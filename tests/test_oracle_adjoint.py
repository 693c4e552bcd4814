"""Pins of the oracle's vector-Jacobian products (CPU only): FD, dot-product, mass invariant."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint, hydro
from paper_2512_13403_b300 import inputs

G = 5.0 / 3.0


def _setup(n=8, steps=4, seed=2, mach=0.8):
    U0 = torch.from_numpy(inputs.decaying_turbulence((n, n, n), seed=seed, sigma=0.3, mach=mach, p_sigma=0.3))
    dx = (1.0 / n,) * 3
    dts = []
    U = U0.clone()
    for _ in range(steps):
        dt = hydro.cfl_dt(U, G, dx, 0.4)
        dts.append(dt)
        U = hydro.rk2_step(U, dt, G, dx)
    return U0, dx, dts


def test_central_finite_differences():
    U0, dx, dts = _setup()
    gen = torch.Generator().manual_seed(0)
    w = torch.randn(U0.shape, generator=gen, dtype=torch.float64)
    loss = lambda U: float((w * adjoint.advance(U, dts, G, dx)).sum())
    g = adjoint.advance_vjp(U0, dts, w, G, dx)
    idx = [(0, 1, 2, 3), (1, 4, 4, 4), (2, 7, 0, 5), (3, 2, 6, 1), (4, 5, 5, 0), (4, 0, 3, 7)]
    for i in idx:
        eps = 1e-6 * max(1.0, abs(float(U0[i])))
        Up = U0.clone(); Up[i] += eps
        Um = U0.clone(); Um[i] -= eps
        fd = (loss(Up) - loss(Um)) / (2 * eps)
        assert fd == pytest.approx(float(g[i]), rel=1e-5, abs=1e-8), i


def test_dot_product_identity():
    U0, dx, dts = _setup(seed=5)
    gen = torch.Generator().manual_seed(1)
    lam = torch.randn(U0.shape, generator=gen, dtype=torch.float64)
    v = torch.randn(U0.shape, generator=gen, dtype=torch.float64)
    # J v by forward-mode AD, J^T lambda by the oracle's reverse product
    _, Jv = torch.func.jvp(lambda U: adjoint.advance(U, dts, G, dx), (U0,), (v,))
    JTl = adjoint.advance_vjp(U0, dts, lam, G, dx)
    a = float((lam * Jv).sum())
    b = float((JTl * v).sum())
    assert a == pytest.approx(b, rel=1e-12)


def test_mass_invariant():
    U0, dx, dts = _setup(seed=7)
    N3 = U0[0].numel()
    lam = torch.zeros_like(U0)
    lam[0] = 1.0 / N3  # L = mean(rho_final)
    g = adjoint.advance_vjp(U0, dts, lam, G, dx)
    assert float((g[0] - 1.0 / N3).abs().max()) < 1e-15
    assert float(g[1:].abs().max()) < 1e-15


def _source_setup(n=8, steps=3, seed=3):
    """Driven, cooling lognormal box recorded through the oracle driver; a small maximum
    fractional change per substep makes dense cells subcycle while others take the trapezoid."""
    from oracle import driver
    U0 = torch.from_numpy(inputs.decaying_turbulence((n, n, n), seed=seed, sigma=0.5, mach=0.8, p_sigma=0.3))
    cfg = driver.Config(shape=(n, n, n), gamma=G, forcing=True, ou_seed=11, cooling=True,
                        t_floor=0.05, cool_frac=0.02)
    sim = driver.Simulation(cfg, U0)
    dts, fields = adjoint.record(sim, steps)
    cool = dict(T_floor=0.05, frac=0.02, nsub_max=1024)
    return U0, cfg.dx, dts, fields, cool


def test_sources_central_finite_differences():
    from oracle import cooling
    U0, dx, dts, fields, cool = _source_setup()
    # both cooling branches occur
    U1 = hydro.rk2_step(U0, dts[0], G, dx)
    rho = U1[0]
    Eth = U1[4] - 0.5 * (U1[1] ** 2 + U1[2] ** 2 + U1[3] ** 2) / rho
    nsub, _ = cooling.substep_count(Eth, rho, dts[0], G, 0.05, 0.02)
    assert bool((nsub == 1).any()) and bool((nsub > 1).any())
    gen = torch.Generator().manual_seed(2)
    w = torch.randn(U0.shape, generator=gen, dtype=torch.float64)
    loss = lambda U: float((w * adjoint.advance(U, dts, G, dx, fields, cool)).sum())
    g = adjoint.advance_vjp(U0, dts, w, G, dx, fields, cool)
    for i in [(0, 1, 2, 3), (1, 4, 4, 4), (2, 7, 0, 5), (3, 2, 6, 1), (4, 5, 5, 0), (4, 0, 3, 7), (0, 6, 1, 1)]:
        eps = 1e-6 * max(1.0, abs(float(U0[i])))
        Up = U0.clone(); Up[i] += eps
        Um = U0.clone(); Um[i] -= eps
        fd = (loss(Up) - loss(Um)) / (2 * eps)
        assert fd == pytest.approx(float(g[i]), rel=1e-5, abs=1e-8), i


def test_sources_mass_invariant():
    """Forcing and cooling leave the density alone: the gradient of the mean final density is
    still exactly 1/N^3 in rho and zero elsewhere."""
    U0, dx, dts, fields, cool = _source_setup(seed=4)
    N3 = U0[0].numel()
    lam = torch.zeros_like(U0)
    lam[0] = 1.0 / N3
    g = adjoint.advance_vjp(U0, dts, lam, G, dx, fields, cool)
    assert float((g[0] - 1.0 / N3).abs().max()) < 1e-15
    assert float(g[1:].abs().max()) < 1e-15


def test_gravity_central_finite_differences_and_mass_invariant():
    from oracle import driver
    n = 8
    # a generic state (every primitive fluctuates): a fluid at rest would put every velocity
    # slope on the limiter's kink, where finite differences see one-sided slopes
    U0 = torch.from_numpy(inputs.decaying_turbulence((n, n, n), seed=5, sigma=0.5, mach=0.8, p_sigma=0.3))
    cfg = driver.Config(shape=(n, n, n), gamma=G, forcing=True, ou_seed=11, cooling=True,
                        t_floor=0.05, cool_frac=0.02, gravity=True, four_pi_G=1.0, mg_tol=1e-12,
                        mg_max_cycles=60)
    sim = driver.Simulation(cfg, U0)
    dts, fields = adjoint.record(sim, 3)
    cool = dict(T_floor=0.05, frac=0.02, nsub_max=1024)
    grav = dict(four_pi_G=1.0)
    dx = cfg.dx
    gen = torch.Generator().manual_seed(3)
    w = torch.randn(U0.shape, generator=gen, dtype=torch.float64)
    loss = lambda U: float((w * adjoint.advance(U, dts, G, dx, fields, cool, grav)).sum())
    g = adjoint.advance_vjp(U0, dts, w, G, dx, fields, cool, grav)
    for i in [(0, 1, 2, 3), (0, 5, 5, 5), (1, 4, 4, 4), (3, 2, 6, 1), (4, 5, 5, 0)]:
        eps = 1e-6 * max(1.0, abs(float(U0[i])))
        Up = U0.clone(); Up[i] += eps
        Um = U0.clone(); Um[i] -= eps
        fd = (loss(Up) - loss(Um)) / (2 * eps)
        assert fd == pytest.approx(float(g[i]), rel=1e-5, abs=1e-8), i
    N3 = n ** 3
    lam = torch.zeros_like(U0)
    lam[0] = 1.0 / N3
    gm = adjoint.advance_vjp(U0, dts, lam, G, dx, fields, cool, grav)
    assert float((gm[0] - 1.0 / N3).abs().max()) < 1e-15
    assert float(gm[1:].abs().max()) < 1e-15
