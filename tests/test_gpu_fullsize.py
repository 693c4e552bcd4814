"""Parity at the measured sizes, in the launch configuration the benchmark times, on sampled
outputs the oracle computes one by one, or through properties that hold at any size.

- Forward step at 256^3 (driven cooling turbulence, float32, forcing and cooling): one step of
  the GPU against the oracle step of a 13^3 periodic block around each sampled cell.  One step
  reaches 4 cells (two stages, each a 2-cell stencil), so a block of 6 cells on each side gives
  the centre exactly.
- Adjoint at 256^3 (decaying turbulence, float32, 20 steps, checkpoint every 10): the gradient
  of the mean final density is exactly 1/N^3 on rho and 0 on the other fields, on any branch.
- Multigrid at 1024^3 (the self-gravitating box, cold solve to 1e-6): the residual F - A phi,
  computed by the oracle's operator at sampled cells from the GPU potential, against rms(F).
- Corrector network at 64^3: the network at sampled cells against the oracle network on a
  13^3 block (three 3x3x3 layers reach 3 cells).
- Self-gravitating step at 1024^3 (lognormal sigma = 1, forcing, cooling, multigrid gravity to
  1e-6): one GPU step against the oracle's step of a 13^3 block around each sampled cell, with
  the potential the GPU solved for (the kick needs it only at the cell's six neighbours; the
  solve itself is checked by the multigrid test).
"""
import math

import numpy as np
import pytest
import torch

from oracle import cooling as ocool
from oracle import corrector as oc
from oracle import forcing as oforce
from oracle import hydro as ohydro
from paper_2512_13403_b300 import inputs
from tests.gpu_util import solver

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _block(U, k, j, i, r):
    """The periodic block of half-width r around cell (k, j, i) of U (5, nz, ny, nx)."""
    nz, ny, nx = U.shape[1:]
    ks = torch.arange(k - r, k + r + 1) % nz
    js = torch.arange(j - r, j + r + 1) % ny
    is_ = torch.arange(i - r, i + r + 1) % nx
    return U[:, ks][:, :, js][:, :, :, is_], (ks, js, is_)


def test_forward_step_256_sampled_cells_vs_oracle():
    n = 256
    shape = (n, n, n)
    dx = (1.0 / n,) * 3
    U0 = inputs.decaying_turbulence(shape, seed=11, sigma=0.5, mach=1.0, P0=0.6)
    U0 = torch.from_numpy(U0).float()            # the float32 state both sides start from
    Ud = U0.double()
    ou = oforce.OUForcing(seed=1, tau=0.5, a_rms=1.0)
    ou.update(1e-3, 0)
    dt = ohydro.cfl_dt(Ud, G, dx, 0.4)
    s = solver(shape, "f32", forcing=True, ou_seed=1, cooling=True, t_floor=0.05)
    s.init_state(U0.cuda().contiguous())
    assert s.compute_dt() == pytest.approx(dt, rel=2e-6)
    s.set_forcing_modes(ou.a_hat.numpy(), hold=True)   # the same table on both sides
    s.step(dt)
    out = s.get_state().cpu().double()
    g = torch.Generator().manual_seed(5)
    samples = torch.randint(0, n, (160, 3), generator=g).tolist()
    samples += [[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, 128]]   # periodic corners
    r = 6
    worst = 0.0
    scale = Ud.abs().amax(dim=(1, 2, 3))
    scale[1:4] = Ud[1:4].abs().max()
    for k, j, i in samples:
        B, (ks, js, is_) = _block(Ud, k, j, i, r)
        kk, jj, ii = torch.meshgrid(ks, js, is_, indexing="ij")
        a = ou.field_at(shape, kk, jj, ii)
        V = ohydro.rk2_step(B, dt, G, dx)
        V = oforce.apply_forcing(V, a, dt)
        V, _ = ocool.cool(V, dt, G, 0.05, 0.1, 1024)
        ref = V[:, r, r, r]
        got = out[:, k, j, i]
        worst = max(worst, float(((got - ref).abs() / scale).max()))
    assert worst < 4e-6, worst


def test_adjoint_256_mass_invariant():
    n = 256
    shape = (n, n, n)
    U0 = inputs.decaying_turbulence(shape, seed=2, sigma=0.5, mach=2.0)
    s = solver(shape, "f32")
    s.init_state(torch.from_numpy(U0).float().cuda().contiguous())
    lam = torch.zeros((5,) + shape, dtype=torch.float32, device="cuda")
    lam[0] = 1.0 / n ** 3
    g = s.adjoint_advance(20, 10, lam)
    err_rho = float((g[0].double() * n ** 3 - 1.0).abs().max())
    err_rest = float(g[1:].double().abs().max()) * n ** 3
    assert err_rho < 2e-5 and err_rest < 2e-5, (err_rho, err_rest)


def test_multigrid_1024_sampled_residual():
    n = 1024
    shape = (n, n, n)
    h = 1.0 / n
    rho = inputs.self_gravitating_box_device(shape, seed=5, sigma=1.0)[0].contiguous()
    s = solver(shape, "f32", gravity=True, four_pi_G=1.0, mg_tol=1e-6, mg_max_cycles=30)
    _, cycles, res = s.solve_poisson(rho, fetch=False)
    assert res <= 1e-6
    rho_h = rho.cpu().numpy()
    del rho
    mean = float(rho_h.mean(dtype=np.float64))
    rmsF = math.sqrt(float(((rho_h.astype(np.float64) - mean) ** 2).mean()))
    phi, _, _ = s.potential()                  # float64 on the device, <phi> = 0
    g = torch.Generator().manual_seed(7)
    idx = torch.randint(0, n, (4096, 3), generator=g)
    k, j, i = idx[:, 0], idx[:, 1], idx[:, 2]
    kd, jd, id_ = k.cuda(), j.cuda(), i.cuda()
    nb = lambda dk, dj, di: phi[(kd + dk) % n, (jd + dj) % n, (id_ + di) % n].cpu()
    c = nb(0, 0, 0)
    lap = (nb(1, 0, 0) + nb(-1, 0, 0) + nb(0, 1, 0) + nb(0, -1, 0) + nb(0, 0, 1) + nb(0, 0, -1)
           - 6.0 * c) / (h * h)
    F = torch.from_numpy(rho_h[k.numpy(), j.numpy(), i.numpy()].astype(np.float64)) - mean
    rel = math.sqrt(float(((F - lap) ** 2).mean())) / rmsF
    # the solver's global relative residual is <= 1e-6; a sample of 4096 cells estimates it
    assert rel < 3e-6, rel
    s.close()


def test_corrector_64_sampled_cells_vs_oracle():
    from paper_2512_13403_b300 import corrector as cr
    n = 64
    shape = (n, n, n)
    p = cr.init_params(4, out_scale=1.0)
    p = p + 0.01 * torch.randn(p.shape, generator=torch.Generator().manual_seed(4))
    pd = cr.unflatten(p.double())
    U = torch.from_numpy(inputs.decaying_turbulence(shape, seed=1, sigma=0.5, mach=1.0, p_sigma=0.3)).float()
    mu = [float(U[c].mean()) for c in range(5)]
    sg = [float(U[c].std()) for c in range(5)]
    net = cr.Network(shape)
    net.set_params(p, mu, sg)
    y = net.forward(U.cuda().contiguous()).cpu().double()
    net.close()
    g = torch.Generator().manual_seed(3)
    samples = torch.randint(0, n, (48, 3), generator=g).tolist() + [[0, 0, 0], [n - 1, 0, n - 1]]
    r = 6
    num = den = 0.0
    Ud = U.double()
    for k, j, i in samples:
        B, _ = _block(Ud, k, j, i, r)
        yr, _ = oc.forward(B, pd, mu, sg)
        d = y[:, k, j, i] - yr[:, r, r, r]
        num += float((d ** 2).sum())
        den += float((yr[:, r, r, r] ** 2).sum())
    assert math.sqrt(num / den) < 1e-2


def test_conserved_totals_256_float32():
    """The float32 state's totals (compensated float32 chunks, float64 across them) against
    float64 sums on the host, at the benchmark's size."""
    n = 256
    shape = (n, n, n)
    U0 = torch.from_numpy(inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=1.0, P0=0.6)).float()
    s = solver(shape, "f32")
    s.init_state(U0.cuda().contiguous())
    tot = s.conserved_totals()
    Uh = U0.numpy().astype(np.float64)
    for f in range(5):
        ref = float(Uh[f].sum())
        scale = float(np.abs(Uh[f]).sum())
        assert abs(tot[f] - ref) <= 1e-12 * scale, (f, tot[f], ref)


def test_self_gravitating_step_1024_sampled_cells_vs_oracle():
    from oracle import multigrid as omg
    n = 1024
    shape = (n, n, n)
    h = 1.0 / n
    dx = (h, h, h)
    s = solver(shape, "f32", forcing=True, ou_seed=3, cooling=True, t_floor=0.05, gravity=True,
               four_pi_G=1.0, mg_tol=1e-6, mg_max_cycles=30)
    U0 = inputs.self_gravitating_box_device(shape, seed=5, sigma=1.0)
    s.init_state(U0)
    del U0
    s.advance(2)                                  # a moving state, and a warm-started solve
    Ub = s.get_state()                            # float32, on the device
    ou = oforce.OUForcing(seed=4, tau=0.5, a_rms=1.0)
    s.set_forcing_modes(ou.a_hat.numpy(), hold=True)   # the same table on both sides
    dt = s.compute_dt()
    s.step(dt)
    out = s.get_state()
    phi, cycles, res = s.potential()              # the solve of this step (float64, <phi> = 0)
    assert res <= 1e-6
    g = torch.Generator().manual_seed(9)
    samples = torch.randint(0, n, (48, 3), generator=g).tolist() + [[0, 0, 0], [n - 1, n - 1, n - 1]]
    r = 6
    scale = torch.stack([Ub[c].abs().max() for c in range(5)]).double().cpu()
    scale[1:4] = scale[1:4].max()
    worst = 0.0
    for k, j, i in samples:
        ks = (torch.arange(k - r, k + r + 1) % n).cuda()
        js = (torch.arange(j - r, j + r + 1) % n).cuda()
        is_ = (torch.arange(i - r, i + r + 1) % n).cuda()
        B = Ub[:, ks][:, :, js][:, :, :, is_].double().cpu()
        P = phi[ks][:, js][:, :, is_].cpu()
        kk, jj, ii = torch.meshgrid(ks.cpu(), js.cpu(), is_.cpu(), indexing="ij")
        V = ohydro.rk2_step(B, dt, G, dx)
        V = oforce.apply_forcing(V, ou.field_at(shape, kk, jj, ii), dt)
        V = omg.gravity_source(V, P, dt, h)
        V, _ = ocool.cool(V, dt, G, 0.05, 0.1, 1024)
        ref = V[:, r, r, r]
        got = out[:, k, j, i].double().cpu()
        worst = max(worst, float(((got - ref).abs() / scale).max()))
    assert worst < 4e-6, worst
    s.close()
