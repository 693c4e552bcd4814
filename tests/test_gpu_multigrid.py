"""GPU multigrid Poisson solve and self-gravity step against the oracle and exact solutions."""
import math

import numpy as np
import pytest
import torch

from oracle import driver as odrv
from oracle import multigrid as omg
from paper_2512_13403_b300 import inputs
from tests.gpu_util import rel_l1, rel_linf, solver, to_gpu

pytestmark = pytest.mark.gpu


def _fft_solution(F, h):
    """Exact solve of the periodic 7-point system: eigenvalue -(4/h^2) sum_a sin^2(pi k_a / n_a)."""
    n = F.shape
    k = [torch.fft.fftfreq(m, d=1.0 / m, dtype=torch.float64) for m in n]
    s = [torch.sin(math.pi * kk / m) ** 2 for kk, m in zip(k, n)]
    lam = -(4.0 / h ** 2) * (s[0][:, None, None] + s[1][None, :, None] + s[2][None, None, :])
    lam[0, 0, 0] = 1.0
    Fh = torch.fft.fftn(F)
    Fh[0, 0, 0] = 0.0
    return torch.fft.ifftn(Fh / lam).real


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_single_fourier_mode(prec):
    n = 32
    h = 1.0 / n
    x = (torch.arange(n, dtype=torch.float64) + 0.5) / n
    m = (1, 2, 3)
    F = torch.sin(2 * math.pi * (m[0] * x[None, None, :] + m[1] * x[None, :, None] + m[2] * x[:, None, None]))
    lam = -(4.0 / h ** 2) * sum(math.sin(math.pi * mi * h) ** 2 for mi in m)
    rho = 1.0 + 0.5 * F  # 4 pi G = 2 gives F back
    s = solver((n, n, n), prec, gravity=True, four_pi_G=2.0, mg_tol=1e-10, mg_max_cycles=40)
    phi, cyc, res = s.solve_poisson(to_gpu(rho.numpy()[None], prec)[0].contiguous())
    exact = F / lam
    tol = 1e-9 if prec == "f64" else 2e-7  # float32 density input rounds F
    assert res <= 1e-10
    assert float((phi.cpu() - exact).abs().max()) < tol * float(exact.abs().max())


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 40), (12, 12, 12)])
def test_matches_fft_solution(shape):
    h = 1.0 / shape[2]
    rho = inputs.lognormal_density(shape, 1.0, 5)
    F = omg.poisson_source(torch.from_numpy(rho), 1.0)
    exact = _fft_solution(F, h)
    s = solver(shape, "f64", gravity=True, dx=(h, h, h), mg_tol=1e-11, mg_max_cycles=60)
    phi, cyc, res = s.solve_poisson(to_gpu(rho[None], "f64")[0].contiguous())
    assert res <= 1e-11
    assert float((phi.cpu() - exact).abs().max()) < 1e-9 * float(exact.abs().max())
    assert abs(float(phi.mean())) < 1e-12 * float(exact.abs().max())


def test_default_tolerance_fp32_residual_and_cycles():
    shape = (64, 64, 64)
    h = 1.0 / 64
    rho = inputs.lognormal_density(shape, 1.0, 7)
    s = solver(shape, "f32", gravity=True)
    rho32 = to_gpu(rho[None], "f32")[0].contiguous()
    phi, cyc, res = s.solve_poisson(rho32)
    # residual checked independently in float64 on the host, for the float32 density given
    F = omg.poisson_source(rho32.double().cpu(), 1.0)
    r = omg.relative_residual(phi.cpu(), F, h)
    assert res <= 1e-6 and r <= 1.000001e-6, (res, r)
    # cycle count comparable to the oracle's V-cycle on the same system
    _, ocyc, ores, ok = omg.solve(F, h, tol=1e-6, max_cycles=30)
    assert ok and abs(cyc - ocyc) <= 2, (cyc, ocyc)


@pytest.mark.parametrize("smoother,cycle_type", [("rbgs", "V"), ("jacobi", "W")])
def test_gravity_step_fp64_vs_oracle(smoother, cycle_type):
    """The float64 context runs the oracle's float64 cycles (same smoother, transfer operators
    and coarse solve), so its iterates, cycle counts and potential follow the oracle's to
    rounding, and the state meets the float64 bar of 1e-11 relative L-infinity."""
    shape = (16, 16, 16)
    U0 = inputs.self_gravitating_box(shape, seed=5, sigma=1.0)
    kw = dict(gravity=True, mg_tol=1e-11, mg_max_cycles=60, mg_smoother=smoother,
              mg_cycle=cycle_type)
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    for _ in range(3):
        dt = s.step(0.0)
        dto = sim.step()
        assert dt == pytest.approx(dto, rel=1e-13)
        phi, cyc, res = s.potential()
        assert cyc == sim.mg_cycles and res <= 1e-11
    assert float((phi.cpu() - sim.phi).abs().max()) < 1e-11 * float(sim.phi.abs().max())
    assert max(rel_linf(s.get_state(), sim.U)) <= 1e-11


@pytest.mark.parametrize("shape", [(32, 32, 32), (8, 12, 64)])
def test_self_gravitating_cooling_turbulence_fp32_vs_oracle(shape):
    """All sources together (forcing, gravity, cooling).  Both sides solve the Poisson problem
    to 1e-10 so that the comparison sees float32 rounding, not two different 1e-6 iterates
    (the default tolerance is covered by test_default_tolerance_fp32_residual_and_cycles).
    Rows of 64 cells take the two-cells-per-thread source kernel, with a ragged last row
    block (12 rows in blocks of 8)."""
    U0 = inputs.self_gravitating_box(shape, seed=5, sigma=1.0)
    h = 1.0 / shape[2]   # cubic cells (gravity needs them) on non-cubic grids
    kw = dict(forcing=True, cooling=True, gravity=True, mg_tol=1e-10, mg_max_cycles=60,
              dx=(h, h, h))
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, "f32", **kw)
    s.init_state(to_gpu(U0, "f32"))
    for _ in range(3):
        dt = s.step(0.0)
        dto = sim.step(dt)
    err = rel_linf(s.get_state(), sim.U)
    assert max(err) < 1e-4, err


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 16, 64)])
def test_smooth_self_gravitating_fp32_50_steps_every_field(shape):
    """The float32 production path with every source (OU forcing, multigrid gravity, cooling)
    on a smooth self-gravitating state (lognormal density, sigma = 0.3) over 50 steps: each
    field within 1e-5 relative L1 of the float64 oracle on its own scale.  Both sides solve the
    Poisson problem to 1e-10, so the comparison sees float32 rounding, not two iterates that
    each stop somewhere within a loose tolerance.  Rows of 64 cells take the two-cells-per-thread
    source kernel (and the paired stage kernel)."""
    U0 = inputs.self_gravitating_box(shape, seed=5, sigma=0.3)
    h = 1.0 / shape[2]   # cubic cells (gravity needs them) on non-cubic grids
    kw = dict(forcing=True, cooling=True, gravity=True, mg_tol=1e-10, mg_max_cycles=60,
              dx=(h, h, h))
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, "f32", **kw)
    s.init_state(to_gpu(U0, "f32"))
    for _ in range(50):
        dt = s.step(0.0)
        dto = sim.step(dt)
    err = rel_l1(s.get_state(), sim.U)
    assert max(err) < 1e-5, err


def test_nonconvergence_is_reported_and_rolled_back():
    from paper_2512_13403_b300._lib import DH_ERR_MG_NOCONV, DhError
    shape = (16, 16, 16)
    U0 = inputs.self_gravitating_box(shape, seed=3, sigma=1.0)
    s = solver(shape, "f64", gravity=True, mg_tol=1e-14, mg_max_cycles=1)
    s.init_state(to_gpu(U0, "f64"))
    with pytest.raises(DhError) as e:
        s.step(0.0)
    assert e.value.status == DH_ERR_MG_NOCONV
    assert torch.equal(s.get_state().cpu(), torch.from_numpy(U0))
    assert s.time() == (0.0, 0)


VARIANTS = [("jacobi", "W"), ("jacobi", "V"), ("rbgs", "W")]


@pytest.mark.parametrize("smoother,cycle_type", VARIANTS)
@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 40), (12, 20, 30)])
def test_variants_match_fft_solution(shape, smoother, cycle_type):
    """Weighted Jacobi (omega = 2/3) and W-cycles (Sec. 5.2, App. C) reach the exact solution of
    the same operator.  (12, 20, 30) has rows of 30 cells, not a multiple of 4 (the
    one-cell-per-thread smoother kernels)."""
    h = 1.0 / shape[2]
    rho = inputs.lognormal_density(shape, 1.0, 5)
    F = omg.poisson_source(torch.from_numpy(rho), 1.0)
    exact = _fft_solution(F, h)
    s = solver(shape, "f64", gravity=True, dx=(h, h, h), mg_tol=1e-11, mg_max_cycles=120,
               mg_smoother=smoother, mg_cycle=cycle_type)
    phi, cyc, res = s.solve_poisson(to_gpu(rho[None], "f64")[0].contiguous())
    assert res <= 1e-11
    assert float((phi.cpu() - exact).abs().max()) < 1e-9 * float(exact.abs().max())


@pytest.mark.parametrize("smoother,cycle_type", VARIANTS + [("rbgs", "V")])
def test_variant_cycle_counts_match_oracle(smoother, cycle_type):
    """The same cycle on both sides contracts at the same rate: equal cycle counts to 1e-8
    (the float32 corrections change the iterates only in the rounding)."""
    shape = (64, 64, 64)
    h = 1.0 / 64
    rho = inputs.lognormal_density(shape, 1.0, 7)
    s = solver(shape, "f64", gravity=True, mg_tol=1e-8, mg_max_cycles=60, mg_smoother=smoother,
               mg_cycle=cycle_type)
    phi, cyc, res = s.solve_poisson(to_gpu(rho[None], "f64")[0].contiguous())
    F = omg.poisson_source(torch.from_numpy(rho), 1.0)
    _, ocyc, ores, ok = omg.solve(F, h, tol=1e-8, max_cycles=60, smoother=smoother,
                                  cycle_type=cycle_type)
    assert ok and res <= 1e-8
    assert abs(cyc - ocyc) <= 1, (cyc, ocyc)


def test_gravity_step_jacobi_wcycle_fp64_vs_oracle():
    shape = (16, 16, 16)
    U0 = inputs.self_gravitating_box(shape, seed=4, sigma=1.0)
    kw = dict(gravity=True, mg_tol=1e-11, mg_max_cycles=120, mg_smoother="jacobi", mg_cycle="W")
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    for _ in range(3):
        dt = s.step(0.0)
        dto = sim.step()
        assert dt == pytest.approx(dto, rel=1e-9)
    phi, cyc, res = s.potential()
    assert float((phi.cpu() - sim.phi).abs().max()) < 1e-8 * float(sim.phi.abs().max())
    assert max(rel_linf(s.get_state(), sim.U)) <= 1e-9


@pytest.mark.parametrize("smoother,cycle_type", [("rbgs", "V"), ("jacobi", "W")])
def test_cycle_graph_on_a_side_stream_matches_direct_launches(smoother, cycle_type):
    """On a stream that can be captured, each cycle replays a CUDA graph; on the legacy default
    stream it cannot be, and the cycle is launched directly.  Same kernels, same order: the
    potentials agree bit for bit, over a cold solve and a warm-started one."""
    from paper_2512_13403_b300.solver import Config, Solver
    shape = (32, 32, 32)
    rho = inputs.lognormal_density(shape, 1.0, 9)
    kw = dict(shape=shape, precision="f64", gravity=True, mg_tol=1e-10, mg_max_cycles=80,
              mg_smoother=smoother, mg_cycle=cycle_type)
    out = []
    for stream in (None, torch.cuda.Stream()):
        with torch.cuda.stream(stream if stream is not None else torch.cuda.default_stream()):
            s = Solver(Config(**kw), stream=stream)
            r = to_gpu(rho[None], "f64")[0].contiguous()
            phi1, c1, _ = s.solve_poisson(r)
            phi2, c2, _ = s.solve_poisson((r * 1.01).contiguous())
            torch.cuda.synchronize()
            out.append((phi1.cpu(), phi2.cpu(), c1, c2))
            s.close()
    (a1, a2, ca1, ca2), (b1, b2, cb1, cb2) = out
    assert (ca1, ca2) == (cb1, cb2)
    assert torch.equal(a1, b1) and torch.equal(a2, b2)


@pytest.mark.parametrize("shape,prec", [((16, 32, 64), "f64"), ((32, 32, 32), "f32"), ((16, 8, 4), "f64")])
def test_fft_poisson_matches_oracle(shape, prec):
    """dh_fft_poisson (exact DFT solve of the same operator) against the oracle's FFT solve."""
    h = 1.0 / shape[2]
    rho = inputs.lognormal_density(shape, 1.0, 4)
    s = solver(shape, prec, gravity=True, dx=(h, h, h), four_pi_G=1.7)
    r = to_gpu(rho[None], prec)[0].contiguous()
    phi = s.fft_poisson(r).cpu()
    F = omg.poisson_source(r.double().cpu(), 1.7)
    exact = omg.fft_solve(F, h)
    assert float((phi - exact).abs().max()) < 1e-12 * float(exact.abs().max())
    s.close()


def test_fft_poisson_agrees_with_multigrid_and_rejects_other_sizes():
    from paper_2512_13403_b300._lib import DH_ERR_ARG, DhError
    shape = (32, 32, 32)
    rho = inputs.lognormal_density(shape, 1.0, 8)
    s = solver(shape, "f64", gravity=True, mg_tol=1e-12, mg_max_cycles=80)
    r = to_gpu(rho[None], "f64")[0].contiguous()
    phi_mg, _, res = s.solve_poisson(r)
    phi_fft = s.fft_poisson(r)
    assert res <= 1e-12
    assert float((phi_mg - phi_fft).abs().max()) < 1e-10 * float(phi_fft.abs().max())
    s.close()
    s = solver((12, 16, 16), "f64", gravity=True, dx=(1 / 16, 1 / 16, 1 / 16))
    with pytest.raises(DhError) as e:
        s.fft_poisson(torch.ones((12, 16, 16), dtype=torch.float64, device="cuda"))
    assert e.value.status == DH_ERR_ARG
    s.close()


def test_cooling_time_step_limit_with_gravity_fp64():
    """With gravity the sources run in their own kernel, which also reduces the next dt: the
    cooling time-step limit there against the oracle."""
    shape = (16, 16, 16)
    U0 = inputs.self_gravitating_box(shape, seed=5, sigma=1.0)
    kw = dict(gravity=True, mg_tol=1e-11, mg_max_cycles=60, cooling=True, t_floor=0.05, c_cool=0.02)
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    for _ in range(3):
        dt = s.step(0.0)
        dto = sim.step()
        assert dt == pytest.approx(dto, rel=1e-9)
    assert max(rel_linf(s.get_state(), sim.U)) <= 1e-9


def test_point_mass_force_multigrid_against_fft():
    """A point mass at the centre (Sec. 5.2's MG-against-FFT comparison): the multigrid force
    g = -grad phi matches the exact DFT solve's to 0.1% of the maximum force at a residual
    tolerance of 1e-2, and much closer at 1e-6."""
    n = 64
    rho = torch.ones((n, n, n), dtype=torch.float32, device="cuda")
    rho[n // 2, n // 2, n // 2] += float(n) ** 3

    def force(phi):
        return [(torch.roll(phi, -1, d) - torch.roll(phi, 1, d)) * (0.5 * n) for d in range(3)]

    ref = None
    for tol, bound in ((1e-2, 1e-3), (1e-6, 1e-5)):
        s = solver((n, n, n), "f32", gravity=True, mg_tol=tol, mg_max_cycles=100)
        if ref is None:
            gf = force(s.fft_poisson(rho))
            ref = (gf, float(torch.sqrt(gf[0] ** 2 + gf[1] ** 2 + gf[2] ** 2).max()))
        s.solve_poisson(rho, fetch=False)
        phi, _, _ = s.potential()
        gm = force(phi)
        err = float(torch.sqrt(sum((gm[d] - ref[0][d]) ** 2 for d in range(3))).max()) / ref[1]
        assert err < bound, (tol, err)
        s.close()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_potential_commutes_with_reflection(axis):
    """The converged potential of a reflected density is the reflected potential.  Reflection
    swaps the red and black cells on even grids, so the Gauss-Seidel iterates differ and only
    the converged solutions agree, to the tolerance."""
    shape = (32, 16, 24)
    d = 2 - axis
    rho = torch.from_numpy(inputs.self_gravitating_box(shape, seed=3, sigma=1.0)[0]).cuda()
    phis = []
    for r in (rho, torch.flip(rho, dims=[d])):
        s = solver(shape, "f64", gravity=True, mg_tol=1e-12, mg_max_cycles=80,
                   dx=(1 / 32, 1 / 32, 1 / 32))
        s.solve_poisson(r.contiguous(), fetch=False)
        phi, _, _ = s.potential()
        phis.append(phi.cpu())
        s.close()
    ref = phis[0]
    assert float((torch.flip(phis[1], dims=[d]) - ref).abs().max()) < 1e-10 * float(ref.abs().max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_cycles_do_not_change_iterates(prec):
    """The host enqueues as many cycles as the previous solve took and reads the residual once;
    cycles enqueued after convergence do nothing.  A converged warm start therefore takes 0
    cycles and leaves phi bit for bit (more cycles enqueued than run, an odd or even number of
    buffer swaps undone), and a solve from the same warm start gives the same iterates and
    count whether its batches are too short (the count predicted 0) or as long as predicted."""
    shape = (32, 32, 32)
    h = 1.0 / 32
    rho_a = inputs.lognormal_density(shape, 1.0, 11)
    rho_b = inputs.lognormal_density(shape, 0.8, 12)
    kw = dict(gravity=True, mg_tol=1e-10 if prec == "f64" else 1e-6, mg_max_cycles=60)
    a = to_gpu(rho_a[None], prec)[0].contiguous()
    b = to_gpu(rho_b[None], prec)[0].contiguous()

    s1 = solver(shape, prec, **kw)
    phi_a, ca, _ = s1.solve_poisson(a)
    assert ca >= 3
    phi_a2, ca2, _ = s1.solve_poisson(a)
    assert ca2 == 0 and torch.equal(phi_a.cpu(), phi_a2.cpu())
    phi_b1, cb1, rb1 = s1.solve_poisson(b)        # predicted 0 cycles: batches of 1, 1, 2, 4, ...

    s2 = solver(shape, prec, **kw)
    s2.solve_poisson(a)
    phi_b2, cb2, rb2 = s2.solve_poisson(b)        # predicted ca cycles
    assert cb1 == cb2 and rb1 == rb2
    assert torch.equal(phi_b1.cpu(), phi_b2.cpu())
    F = omg.poisson_source(b.double().cpu(), 1.0)
    assert omg.relative_residual(phi_b1.cpu(), F, h) <= kw["mg_tol"] * 1.000001
