"""Pins of the oracle's multigrid Poisson solver and gravity source (CPU only)."""
import math

import numpy as np
import pytest
import torch

from oracle import multigrid as mg
from paper_2512_13403_b300 import inputs


def _coords(shape):
    nz, ny, nx = shape
    return [(torch.arange(n, dtype=torch.float64) + 0.5) / n for n in (nx, ny, nz)]


def test_single_fourier_mode_exact_discrete_solution():
    n = 32
    h = 1.0 / n
    x, y, z = _coords((n, n, n))
    m = (1, 2, 3)
    F = torch.sin(2 * math.pi * (m[0] * x[None, None, :] + m[1] * y[None, :, None] + m[2] * z[:, None, None]))
    lam = -(4.0 / h ** 2) * sum(math.sin(math.pi * mi * h) ** 2 for mi in m)
    phi, cycles, res, ok = mg.solve(F, h, tol=1e-11, max_cycles=40)
    assert ok
    assert float((phi - F / lam).abs().max()) < 1e-9 * float((F / lam).abs().max())


def test_matches_fft_solve_of_same_operator():
    n = 32
    h = 1.0 / n
    rho = torch.from_numpy(inputs.lognormal_density((n, n, n), 1.0, 5))
    F = mg.poisson_source(rho, 1.0)
    k = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64)
    s = lambda kk: torch.sin(math.pi * kk * h) ** 2
    lam = -(4.0 / h ** 2) * (s(k)[:, None, None] + s(k)[None, :, None] + s(k)[None, None, :])
    lam[0, 0, 0] = 1.0
    Fh = torch.fft.fftn(F)
    Fh[0, 0, 0] = 0.0
    phi_fft = torch.fft.ifftn(Fh / lam).real
    phi, cycles, res, ok = mg.solve(F, h, tol=1e-12, max_cycles=60)
    assert ok
    assert float((phi - phi_fft).abs().max()) < 1e-10 * float(phi_fft.abs().max())


def test_vcycle_reduces_residual():
    n = 32
    h = 1.0 / n
    F = mg.poisson_source(torch.from_numpy(inputs.lognormal_density((n, n, n), 1.0, 6)), 1.0)
    shapes = mg.level_shapes(F.shape)
    assert shapes[-1] == (4, 4, 4)
    phi = torch.zeros_like(F)
    r0 = mg.relative_residual(phi, F, h)
    factors = []
    for _ in range(5):
        phi = mg.vcycle(phi, F, h, shapes)
        phi = phi - phi.mean()
        r1 = mg.relative_residual(phi, F, h)
        factors.append(r1 / r0)
        r0 = r1
    assert max(factors) < 0.2, factors


def test_coarse_pseudo_inverse_projects_mean():
    shape = (4, 4, 4)
    F = torch.randn(shape, dtype=torch.float64)
    phi = mg.coarse_solve(F, 0.25)
    assert float(phi.mean().abs()) < 1e-13
    assert torch.allclose(mg.apply_A(phi, 0.25), F - F.mean(), atol=1e-12)


def test_transfer_operators_on_constants_and_linear_fields():
    c = torch.full((4, 6, 8), 2.5, dtype=torch.float64)
    assert torch.allclose(mg.restrict(torch.full((8, 12, 16), 2.5, dtype=torch.float64)), c)
    assert torch.allclose(mg.prolong(c), torch.full((8, 12, 16), 2.5, dtype=torch.float64))
    # a field linear in x (cell-centre coordinates) is reproduced away from the periodic seam
    xc = (torch.arange(8, dtype=torch.float64) + 0.5) / 8
    e = xc[None, None, :].expand(4, 4, 8).contiguous()
    xf = (torch.arange(16, dtype=torch.float64) + 0.5) / 16
    p = mg.prolong(e)
    assert torch.allclose(p[..., 1:-1], xf[None, None, 1:-1].expand(8, 8, 14))
    # restriction after prolongation reproduces a linear field away from the seam
    assert torch.allclose(mg.restrict(p)[..., 1:-1], e[..., 1:-1])


def test_gravity_source_on_linear_potential():
    n = 8
    h = 1.0 / n
    U = torch.from_numpy(inputs.uniform_state((n, n, n), rho=2.0, P=1.0, v=(0.1, 0.0, 0.0)))
    x = (torch.arange(n, dtype=torch.float64) + 0.5) * h
    phi = torch.sin(2 * math.pi * x)[None, None, :].expand(n, n, n).contiguous()
    out = mg.gravity_source(U, phi, 0.01, h)
    gx = -(torch.sin(2 * math.pi * (x + h)) - torch.sin(2 * math.pi * (x - h))) / (2 * h)
    assert torch.allclose(out[1], U[1] + 2.0 * gx[None, None, :] * 0.01, rtol=1e-14)
    assert torch.allclose(out[4], U[4] + U[1] * gx[None, None, :] * 0.01, rtol=1e-14)
    assert torch.equal(out[2], U[2]) and torch.equal(out[0], U[0])


def test_fft_solve_single_mode_and_multigrid():
    nz, ny, nx = 8, 16, 32
    h = 1.0 / 32
    shape = (nz, ny, nx)
    x = (torch.arange(nx, dtype=torch.float64) + 0.5) / nx
    y = (torch.arange(ny, dtype=torch.float64) + 0.5) / ny
    z = (torch.arange(nz, dtype=torch.float64) + 0.5) / nz
    m = (3, 1, 2)   # (x, y, z) wave numbers
    F = torch.cos(2 * math.pi * (m[0] * x[None, None, :] + m[1] * y[None, :, None] + m[2] * z[:, None, None]))
    lam = -(4.0 / h ** 2) * (math.sin(math.pi * m[0] / nx) ** 2 + math.sin(math.pi * m[1] / ny) ** 2 +
                             math.sin(math.pi * m[2] / nz) ** 2)
    phi = mg.fft_solve(F, h)
    assert float((phi - F / lam).abs().max()) < 1e-12 * float((F / lam).abs().max())
    rho = torch.from_numpy(inputs.lognormal_density((16, 16, 16), 1.0, 8))
    F2 = mg.poisson_source(rho, 1.0)
    phi_mg, _, _, ok = mg.solve(F2, 1.0 / 16, tol=1e-12, max_cycles=60)
    assert ok
    phi_f = mg.fft_solve(F2, 1.0 / 16)
    assert float((phi_mg - phi_f).abs().max()) < 1e-10 * float(phi_f.abs().max())


@pytest.mark.parametrize("omega", [2.0 / 3.0, 1.0, 0.5])
def test_weighted_jacobi_amplifies_a_fourier_mode_by_its_symbol(omega):
    """Weighted Jacobi phi + omega D^-1 (F - A phi), D = -6/h^2 (Sec. 5.2), on F = 0 multiplies a
    discrete Fourier mode by 1 - omega + (omega/3) sum_a cos(2 pi m_a / n_a).  (The printed
    component form's (1 - omega)/6 coefficient would give a different factor.)"""
    shape = (8, 12, 16)   # (nz, ny, nx)
    h = 1.0 / 16
    m = (3, 2, 1)         # (m_x, m_y, m_z)
    nz, ny, nx = shape
    i = torch.arange(nx, dtype=torch.float64)[None, None, :]
    j = torch.arange(ny, dtype=torch.float64)[None, :, None]
    k = torch.arange(nz, dtype=torch.float64)[:, None, None]
    phi = torch.cos(2 * math.pi * (m[0] * i / nx + m[1] * j / ny + m[2] * k / nz) + 0.3)
    out = mg.jacobi_sweep(phi, torch.zeros_like(phi), h, omega)
    sym = 1 - omega + omega / 3 * (math.cos(2 * math.pi * m[0] / nx) + math.cos(2 * math.pi * m[1] / ny)
                                   + math.cos(2 * math.pi * m[2] / nz))
    assert float((out - sym * phi).abs().max()) < 1e-13
    # and the source enters as -omega h^2 F / 6
    F = torch.rand(shape, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    out = mg.jacobi_sweep(torch.zeros_like(F), F, h, omega)
    assert float((out + omega * h * h / 6 * F).abs().max()) < 1e-15


@pytest.mark.parametrize("smoother", ["rbgs", "jacobi"])
def test_wcycle_on_two_levels_is_the_vcycle(smoother):
    """Above an exactly solved coarsest level there is nothing to visit twice (App. C)."""
    n = 8
    h = 1.0 / n
    F = mg.poisson_source(torch.from_numpy(inputs.lognormal_density((n, n, n), 1.0, 3)), 1.0)
    shapes = mg.level_shapes(F.shape)
    assert len(shapes) == 2
    phi = 0.01 * F
    v = mg.cycle(phi, F, h, shapes, smoother=smoother, gamma=1)
    w = mg.cycle(phi, F, h, shapes, smoother=smoother, gamma=2)
    assert torch.equal(v, w)


@pytest.mark.parametrize("smoother", ["rbgs", "jacobi"])
def test_wcycle_contracts_faster_than_vcycle_and_visits_levels_twice(smoother):
    n = 32
    h = 1.0 / n
    F = mg.poisson_source(torch.from_numpy(inputs.lognormal_density((n, n, n), 1.0, 6)), 1.0)
    shapes = mg.level_shapes(F.shape)
    assert len(shapes) == 4

    def rate(gamma):
        phi = torch.zeros_like(F)
        r = [mg.relative_residual(phi, F, h)]
        for _ in range(4):
            phi = mg.cycle(phi, F, h, shapes, smoother=smoother, gamma=gamma)
            r.append(mg.relative_residual(phi - phi.mean(), F, h))
        return r[1] / r[4]   # reduction over the last three cycles

    assert rate(2) > 1.2 * rate(1)
    # the W recursion visits level l 2^l times (the coarsest as often as its parent)
    calls = []
    orig = mg.coarse_solve

    def counting(Fc, hc):
        calls.append(Fc.shape)
        return orig(Fc, hc)

    mg.coarse_solve = counting
    try:
        mg.cycle(torch.zeros_like(F), F, h, shapes, smoother=smoother, gamma=2)
    finally:
        mg.coarse_solve = orig
    assert len(calls) == 4   # levels 0, 1, 2 visited 1, 2, 4 times; level 3 once per visit of 2


@pytest.mark.parametrize("smoother,cycle_type", [("jacobi", "W"), ("jacobi", "V"), ("rbgs", "W")])
def test_smoother_and_cycle_variants_reach_the_fft_solution(smoother, cycle_type):
    n = 16
    h = 1.0 / n
    F = mg.poisson_source(torch.from_numpy(inputs.lognormal_density((n, n, n), 1.0, 2)), 1.0)
    phi, cycles, res, ok = mg.solve(F, h, tol=1e-12, max_cycles=80, smoother=smoother,
                                    cycle_type=cycle_type)
    exact = mg.fft_solve(F, h)
    assert ok
    assert float((phi - exact).abs().max()) < 1e-10 * float(exact.abs().max())
