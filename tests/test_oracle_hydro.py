"""Pins of the oracle's hydro scheme against facts fixed outside the oracle (CPU only)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import hydro
from paper_2512_13403_b300 import inputs
from tests import exact_riemann

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _face(W):
    return torch.tensor(W, dtype=torch.float64).reshape(5, 1, 1, 1)


def test_eos_round_trip():
    U = torch.from_numpy(inputs.decaying_turbulence((8, 8, 8), seed=3))
    W = hydro.cons_to_prim(U, 5.0 / 3.0)
    U2 = hydro.prim_to_cons(W, 5.0 / 3.0)
    assert torch.allclose(U2, U, rtol=1e-14, atol=1e-14)
    # P = (gamma-1)(E - rho|v|^2/2) for a hand state: rho=2, v=(1,2,2), E=10, gamma=1.4
    Uh = torch.tensor([2.0, 2.0, 4.0, 4.0, 10.0], dtype=torch.float64).reshape(5, 1, 1, 1)
    Wh = hydro.cons_to_prim(Uh, 1.4).reshape(5)
    assert Wh.tolist() == pytest.approx([2.0, 1.0, 2.0, 2.0, 0.4 * (10.0 - 9.0)], rel=1e-15)


@pytest.mark.parametrize("a,b,expected", [
    (1.0, 1.0, 1.0),        # 1/2|a+b| = 1 = min
    (1.0, -1.0, 0.0),       # extremum
    (0.0, 2.0, 0.0),        # a*b = 0
    (1.0, 3.0, 2.0),        # 2|a| = 2 < 1/2|a+b| = 2 -> tie, 2
    (1.0, 10.0, 2.0),       # 2|a| smallest
    (10.0, 1.0, 2.0),       # 2|b| smallest
    (-3.0, -2.0, -2.5),     # central branch, negative sign
    (-1.0, -4.0, -2.0),     # 2|a| branch, negative
    (2.0, 2.5, 2.25),       # central branch
])
def test_mc_truth_table(a, b, expected):
    got = hydro.mc_limiter(torch.tensor([a], dtype=torch.float64), torch.tensor([b], dtype=torch.float64))
    assert float(got) == expected


def test_hllc_hand_cases():
    with open(os.path.join(GOLDEN, "hllc_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        F = hydro.hllc_flux(_face(c["WL"]), _face(c["WR"]), c["axis"], c["gamma"]).reshape(5)
        assert F.tolist() == pytest.approx(c["F"], abs=1e-13), c["name"]


def test_hllc_consistency_and_rotation():
    rng = np.random.default_rng(7)
    W = torch.from_numpy(np.stack([rng.uniform(0.5, 2, 50), rng.normal(0, 1, 50), rng.normal(0, 1, 50),
                                   rng.normal(0, 1, 50), rng.uniform(0.5, 2, 50)])).reshape(5, 50, 1, 1)
    for axis in range(3):
        F = hydro.hllc_flux(W, W, axis, 1.4)
        assert torch.allclose(F, hydro.physical_flux(W, axis, 1.4), rtol=1e-13, atol=1e-13)
    WR = W.flip(1)
    Fx = hydro.hllc_flux(W, WR, 0, 1.4)
    # permute velocity components x->y, y->z, z->x and evaluate along y
    perm = [0, 3, 1, 2, 4]
    Fy = hydro.hllc_flux(W[perm], WR[perm], 1, 1.4)
    assert torch.allclose(Fy, Fx[perm], rtol=1e-13, atol=1e-13)


def test_hllc_matches_godunov_to_second_order_in_jump():
    """Approximate and exact Riemann fluxes agree up to O(jump^2) (Toro Ch. 10)."""
    g = 1.4
    base = np.array([1.0, 0.3, 0.0, 0.0, 1.0])
    direction = np.array([0.7, -0.4, 0.0, 0.0, 0.9])
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        WL = base - eps * direction
        WR = base + eps * direction
        F = hydro.hllc_flux(_face(WL), _face(WR), 0, g).reshape(5).numpy()
        G = exact_riemann.godunov_flux((WL[0], WL[1], WL[4]), (WR[0], WR[1], WR[4]), g)
        errs.append(max(abs(F[0] - G[0]), abs(F[1] - G[1]), abs(F[4] - G[2])))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.8, (errs, rates)


def _run(U, gamma, t_end, cfl=0.4):
    U = torch.from_numpy(U)
    nz, ny, nx = U.shape[1:]
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    t = 0.0
    while t < t_end - 1e-15:
        dt = min(hydro.cfl_dt(U, gamma, dx, cfl), t_end - t)
        U = hydro.rk2_step(U, dt, gamma, dx)
        t += dt
    return U


def test_double_sod_matches_exact_solution():
    g = 1.4
    errs = []
    for nx in (64, 128, 256):
        U = _run(inputs.double_sod(nx, 2, 2, gamma=g), g, 0.1)
        rho = U[0, 0, 0].numpy()
        x = (np.arange(nx) + 0.5) / nx
        exact = np.empty(nx)
        inner, outer = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
        for i, xi in enumerate(x):
            if xi >= 0.5:
                exact[i] = exact_riemann.sample(inner, outer, g, (xi - 0.75) / 0.1)[0]
            else:
                exact[i] = exact_riemann.sample(outer, inner, g, (xi - 0.25) / 0.1)[0]
        errs.append(np.abs(rho - exact).mean())
        # symmetric in y and z
        assert torch.allclose(U[0], U[0, :1, :1].expand_as(U[0]))
    assert errs[0] < 0.02 and errs[1] < errs[0] and errs[2] < errs[1], errs


def test_sound_wave_second_order():
    g = 1.4
    errs = []
    for nx in (16, 32, 64, 128):
        U0 = inputs.sound_wave(nx, 2, 2, amp=1e-6, gamma=g)
        U = _run(U0, g, 1.0)  # one period: c0 = 1, L = 1
        errs.append(float((U[0] - torch.from_numpy(U0[0])).abs().mean()) / 1e-6)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert rates[-1] > 1.7 and rates[-2] > 1.7, (errs, rates)


def test_conservation_to_roundoff():
    U0 = torch.from_numpy(inputs.kelvin_helmholtz((12, 16, 20), seed=0))
    dx = (1 / 20, 1 / 16, 1 / 12)
    U = U0
    for _ in range(10):
        U = hydro.rk2_step(U, hydro.cfl_dt(U, 5 / 3, dx, 0.4), 5 / 3, dx)
    t0 = hydro.conserved_totals(U0)
    t1 = hydro.conserved_totals(U)
    for f in range(5):
        scale = float(U0[f].abs().sum()) + float(U[f].abs().sum()) + float(U0[4].abs().sum()) * 1e-3
        assert abs(t1[f] - t0[f]) <= 1e-13 * scale, (f, t1[f] - t0[f], scale)


def test_axis_permutation_symmetry():
    """Swapping x and y in the initial state swaps them in the result."""
    U = torch.from_numpy(inputs.decaying_turbulence((8, 12, 12), seed=4, mach=0.5))
    dx = (1 / 12, 1 / 12, 1 / 8)
    A = hydro.rk2_step(U, 1e-3, 5 / 3, dx)
    Us = U[[0, 2, 1, 3, 4]].transpose(2, 3)
    B = hydro.rk2_step(Us, 1e-3, 5 / 3, dx)[[0, 2, 1, 3, 4]].transpose(2, 3)
    assert torch.allclose(A, B, rtol=1e-12, atol=1e-13)


def test_cfl_dt_hand_value():
    g = 5 / 3
    U = torch.from_numpy(inputs.uniform_state((4, 4, 8), rho=2.0, P=3.0, v=(0.5, -1.0, 0.25), gamma=g))
    c = math.sqrt(g * 3.0 / 2.0)
    dx = (1 / 8, 1 / 4, 1 / 4)
    expect = 0.4 * min(dx[0] / (0.5 + c), dx[1] / (1.0 + c), dx[2] / (0.25 + c))
    assert hydro.cfl_dt(U, g, dx, 0.4) == pytest.approx(expect, rel=1e-15)


def test_conserved_totals_exact_sum():
    U = torch.from_numpy(inputs.kelvin_helmholtz((4, 8, 8)))
    tot = hydro.conserved_totals(U)
    assert tot[0] == math.fsum(U[0].reshape(-1).tolist())
    # rho = 2 on half of the y rows, 1 on the other half
    assert tot[0] == 4 * 8 * (4 * 2.0 + 4 * 1.0)


@pytest.mark.parametrize("a,b,expected", [
    (1.0, 3.0, 1.5), (3.0, 1.0, 1.5), (-2.0, -2.0, -2.0), (1.0, -1.0, 0.0), (0.0, 5.0, 0.0),
    (-4.0, -1.0, -1.6), (2.0, 0.0, 0.0)])
def test_van_leer_truth_table(a, b, expected):
    """2ab/(a+b) on same-sign differences, else 0 (the van Leer slope of App. A.1)."""
    got = hydro.van_leer_limiter(torch.tensor([a], dtype=torch.float64), torch.tensor([b], dtype=torch.float64))
    assert float(got) == pytest.approx(expected, abs=1e-15)


def test_van_leer_is_tvd_bounded_and_between_minmod_and_mc():
    rng = np.random.default_rng(3)
    a = torch.from_numpy(rng.normal(size=4000))
    b = torch.from_numpy(rng.normal(size=4000))
    vl = hydro.van_leer_limiter(a, b)
    mc = hydro.mc_limiter(a, b)
    same = a * b > 0
    minmod = torch.where(same, torch.sign(a) * torch.minimum(a.abs(), b.abs()), torch.zeros_like(a))
    assert torch.all(vl.abs() <= 2 * torch.minimum(a.abs(), b.abs()) + 1e-15)
    assert torch.all(vl.abs() >= minmod.abs() - 1e-15)
    assert torch.all(vl.abs() <= mc.abs() + 1e-15)
    # gradients stay finite where a = -b (the branch not taken has a zero denominator)
    x = torch.tensor([1.0, -2.0], dtype=torch.float64, requires_grad=True)
    y = torch.tensor([-1.0, 2.0], dtype=torch.float64, requires_grad=True)
    hydro.van_leer_limiter(x, y).sum().backward()
    assert torch.all(torch.isfinite(x.grad)) and torch.all(x.grad == 0)


@pytest.mark.parametrize("z", [-0.3, -1.0, -2.5, 0.7])
def test_ssprk3_stability_polynomial(z):
    """On dU/dt = lambda U the Shu-Osher SSPRK3 step multiplies by 1 + z + z^2/2 + z^3/6,
    z = lambda dt: the third-order Taylor polynomial (App. A.3 lists SSPRK3)."""
    lam = torch.tensor([[z, 0.4], [-0.4, z]], dtype=torch.float64)   # a rotation-damping pair
    U = torch.tensor([1.0, -0.5], dtype=torch.float64)
    out = hydro.ssprk3(lambda V: lam @ V, U, 1.0)
    P = torch.eye(2, dtype=torch.float64) + lam + lam @ lam / 2 + lam @ lam @ lam / 6
    assert torch.allclose(out, P @ U, rtol=0, atol=1e-15)


@pytest.mark.parametrize("integrator,limiter", [("rk2", "vanleer"), ("ssprk3", "mc"), ("ssprk3", "vanleer")])
def test_variants_sound_wave_second_order_and_conservative(integrator, limiter):
    g = 1.4
    errs = []
    for nx in (16, 32, 64):
        U0 = inputs.sound_wave(nx, 2, 2, amp=1e-6, gamma=g)
        U = torch.from_numpy(U0)
        dx = (1.0 / nx, 1.0 / 2, 1.0 / 2)
        nsteps = int(math.ceil(1.0 / (0.4 / nx)))
        dt = 1.0 / nsteps
        for _ in range(nsteps):
            U = hydro.step(U, dt, g, dx, integrator, limiter)
        errs.append(float((U[0] - torch.from_numpy(U0[0])).abs().mean()) / 1e-6)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > 1.7, (errs, rates)
    U0 = torch.from_numpy(inputs.kelvin_helmholtz((8, 12, 16), seed=0))
    dxk = (1 / 16, 1 / 12, 1 / 8)
    U1 = hydro.step(U0, 1e-3, 5 / 3, dxk, integrator, limiter)
    t0, t1 = hydro.conserved_totals(U0), hydro.conserved_totals(U1)
    for f in range(5):
        assert abs(t1[f] - t0[f]) <= 1e-13 * (float(U0[f].abs().sum()) + float(U0[4].abs().sum()) * 1e-3)
