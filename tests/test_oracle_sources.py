"""Pins of the oracle's OU forcing and cooling source terms (CPU only)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import cooling, forcing
from paper_2512_13403_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64.json")) as f:
        g = json.load(f)
    got = [forcing.stream_word(g["seed_state"], i) for i in range(5)]
    assert got == [int(x) for x in g["outputs"]]


def test_box_muller_moments():
    xs = torch.cat([forcing.gaussian_draw(11, d).reshape(-1) for d in range(200)])
    re = torch.cat([xs.real, xs.imag])
    n = re.numel()  # 19200 samples
    assert abs(float(re.mean())) < 4.0 / math.sqrt(n)
    assert abs(float(re.var()) - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(float((re ** 4).mean()) - 3.0) < 0.15


def test_forced_modes_band():
    modes = forcing.forced_modes()
    full = set()
    for n in modes:
        full.add(n)
        full.add(tuple(-c for c in n))
    brute = {(a, b, c) for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)
             if 1 <= a * a + b * b + c * c <= 4}
    assert full == brute and len(modes) == 16


def test_ou_field_parseval_divergence_mean():
    ou = forcing.OUForcing(seed=1, tau=0.5, a_rms=1.0)
    for s in range(3):
        ou.update(0.01, s)
    shape = (8, 10, 12)
    a = ou.raw_field(shape)
    brute = float((a * a).sum(0).mean())
    assert brute == pytest.approx(ou.mean_square(), rel=1e-12)
    n = torch.tensor(forcing.forced_modes(), dtype=torch.float64).to(torch.complex128)
    assert float((n * ou.a_hat).sum(1).abs().max()) < 1e-14
    assert float(a.mean(dim=(1, 2, 3)).abs().max()) < 1e-14
    an = ou.field(shape)
    assert float((an * an).sum(0).mean()) == pytest.approx(1.0, rel=1e-12)
    # spectral divergence: the discrete central-difference free part is checked via FFT
    A = torch.fft.fftn(a, dim=(1, 2, 3))
    kz = torch.fft.fftfreq(8, dtype=torch.float64) * 8
    ky = torch.fft.fftfreq(10, dtype=torch.float64) * 10
    kx = torch.fft.fftfreq(12, dtype=torch.float64) * 12
    div = kx[None, None, :] * A[0] + ky[None, :, None] * A[1] + kz[:, None, None] * A[2]
    assert float(div.abs().max()) < 1e-10 * float(A.abs().max())


@pytest.mark.slow
def test_ou_stationary_variance():
    """The recurrence keeps the stationary second moment E|a_hat|^2 of the projected draw."""
    ou = forcing.OUForcing(seed=3, tau=0.5, a_rms=1.0)
    acc = 0.0
    nsteps = 3000
    for s in range(nsteps):
        ou.update(0.05, s)
        acc += float((ou.a_hat.abs() ** 2).sum())
    mean = acc / nsteps
    # 16 modes, complex 3-vectors with unit-variance parts projected onto a 2D plane: 16 * 2 * 2
    expect = 64.0
    # correlation time tau/dt = 10 steps -> ~nsteps/20 independent samples of a chi^2_64-like sum
    assert abs(mean - expect) < 5.0 * expect * math.sqrt(2.0 / 64.0) / math.sqrt(nsteps / 20.0)


def test_forcing_kick_from_rest():
    U = torch.from_numpy(inputs.lognormal_density((6, 6, 6), 0.5, 1)[None].repeat(5, 0))
    U[1:4] = 0.0
    U[4] = 3.0
    a = torch.randn(3, 6, 6, 6, dtype=torch.float64)
    out = forcing.apply_forcing(U, a, 0.01)
    assert torch.equal(out[1:4], U[0] * a * 0.01)
    assert torch.equal(out[4], U[4])
    assert torch.equal(out[0], U[0])


def _cell(rho, Eth, m=(0.0, 0.0, 0.0)):
    U = torch.zeros(5, 1, 1, 1, dtype=torch.float64)
    U[0] = rho
    U[1], U[2], U[3] = m
    U[4] = Eth + 0.5 * (m[0] ** 2 + m[1] ** 2 + m[2] ** 2) / rho
    return U


def _closed_form(E0, rho, gamma, t):
    """dE/dt = -rho^2 sqrt((gamma-1)E/rho) = -c sqrt(E): sqrt(E(t)) = sqrt(E0) - c t / 2."""
    c = rho * rho * math.sqrt((gamma - 1.0) / rho)
    return (math.sqrt(E0) - 0.5 * c * t) ** 2


def test_cooling_subcycle_converges_to_closed_form():
    gamma, rho, E0, dt = 5 / 3, 2.0, 1.5, 0.2
    exact = _closed_form(E0, rho, gamma, dt)
    errs = []
    for frac in (0.1, 0.05, 0.025, 0.0125):
        out, _ = cooling.cool(_cell(rho, E0), dt, gamma, 1e-8, frac=frac)
        errs.append(abs(float(out[4]) - exact))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(0.8 < r < 1.2 for r in rates), (errs, rates)  # explicit substeps: first order


def test_cooling_trapezoid_third_order_local_error():
    gamma, rho, E0 = 5 / 3, 1.0, 0.9
    errs = []
    for dt in (1e-2, 5e-3, 2.5e-3):
        out, _ = cooling.cool(_cell(rho, E0), dt, gamma, 1e-8)
        nsub, _ = cooling.substep_count(torch.tensor(E0), torch.tensor(rho), dt, gamma, 1e-8)
        assert float(nsub) == 1.0
        errs.append(abs(float(out[4]) - _closed_form(E0, rho, gamma, dt)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.7, (errs, rates)


def test_cooling_floor_kinetic_and_cold_cells():
    gamma, T_floor = 5 / 3, 0.05
    m = (0.3, -0.2, 0.1)
    U = torch.cat([_cell(4.0, 2.0, m), _cell(1.0, 0.5 * T_floor / (gamma - 1.0), m)], dim=1)
    kin = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    out, cap = cooling.cool(U, 10.0, gamma, T_floor)
    Eth = out[4] - kin
    floor = U[0] * T_floor / (gamma - 1.0)
    assert float(Eth[0]) >= float(floor[0]) - 1e-15
    assert float(Eth[0]) == pytest.approx(float(floor[0]), rel=1e-12)  # long step: reaches the floor
    assert torch.equal(out[4, 1], U[4, 1])  # below the floor: untouched
    assert torch.equal(out[:4], U[:4])


def test_forcing_field_at_cells_equals_the_whole_field():
    from oracle import forcing as of
    ou = of.OUForcing(seed=3, tau=0.5, a_rms=1.0)
    ou.update(0.01, 0)
    shape = (6, 7, 8)
    full = ou.field(shape)
    g = torch.Generator().manual_seed(0)
    k = torch.randint(0, 6, (50,), generator=g)
    j = torch.randint(0, 7, (50,), generator=g)
    i = torch.randint(0, 8, (50,), generator=g)
    assert torch.allclose(ou.field_at(shape, k, j, i), full[:, k, j, i], rtol=0, atol=1e-14)


def test_min_cooling_time_hand_values():
    """t_cool = E_th / |Edot| with Edot = -rho^2 T^(1/2), T = (gamma - 1) E_th / rho (Sec. 4.3),
    evaluated by hand; cells at or below the floor do not count, and with none cooling the
    minimum is +inf.  The cooling limit of the step is then c_cool times that minimum."""
    from oracle import driver, hydro
    g = 5.0 / 3.0
    shape = (4, 4, 4)
    z = np.zeros(shape)
    rho = np.ones(shape)
    P = np.full(shape, 0.6)
    rho[1, 2, 3] = 2.0                   # T = 0.3, E_th = 0.9: t = 0.9 / (4 sqrt(0.3))
    vx = z.copy()
    vx[1, 2, 3] = 0.5                    # kinetic energy does not enter E_th
    U = torch.from_numpy(inputs.prim_to_state(rho, vx, z, z, P, g))
    t = cooling.min_cooling_time(U, g, 0.05)
    assert t == pytest.approx(0.9 / (4.0 * math.sqrt(0.3)), rel=1e-14)
    assert 0.9 / math.sqrt(0.6) > t      # the uniform cells' time is the larger one
    # at the floor (T = T_floor) nothing cools
    U_cold = torch.from_numpy(inputs.prim_to_state(np.ones(shape), z, z, z, np.full(shape, 0.05), g))
    assert cooling.min_cooling_time(U_cold, g, 0.05) == math.inf
    # the step takes min(CFL step, c_cool min t_cool, dt_max)
    sim = driver.Simulation(driver.Config(shape=shape, cooling=True, t_floor=0.05, c_cool=0.01), U)
    cfl = hydro.cfl_dt(U, g, sim.cfg.dx, 0.4)
    assert sim.compute_dt() == pytest.approx(min(cfl, 0.01 * t), rel=1e-15)
    assert 0.01 * t < cfl                # the cooling limit binds here
