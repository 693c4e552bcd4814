"""GPU hand adjoint (dh_adjoint_advance) against the oracle's reverse-mode product, finite
differences of the GPU forward, the dot-product identity and the exact mass invariant.

Derivative checks use generic states (every primitive field fluctuates).  A field that is
exactly uniform puts every slope of that field on the MC limiter's kink (a = b = 0 up to
round-off), where the step has no Jacobian: the branch is then picked by round-off, which the
GPU (fused multiply-adds) and the CPU oracle resolve differently, and finite differences see a
direction-dependent slope.  Uniform fields are exercised by the mass invariant, which holds on
any branch."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import hydro as ohydro
from paper_2512_13403_b300 import inputs
from tests.gpu_util import solver, to_gpu

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _dx(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


def _oracle_dts(U0, shape, n):
    U = torch.from_numpy(U0)
    dts = []
    for _ in range(n):
        dt = ohydro.cfl_dt(U, G, _dx(shape), 0.4)
        dts.append(dt)
        U = ohydro.rk2_step(U, dt, G, _dx(shape))
    return dts


def _rel(a, b):
    a = torch.as_tensor(a).double().cpu()
    b = torch.as_tensor(b).double().cpu()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("shape,n,k", [((16, 16, 16), 6, 4), ((12, 10, 20), 5, 2), ((9, 12, 40), 3, 3),
                                       ((4, 6, 5), 3, 2), ((6, 5, 4), 2, 1)])
def test_fp64_matches_oracle_vjp_smooth(shape, n, k):
    U0 = inputs.decaying_turbulence(shape, seed=5, sigma=0.3, mach=0.8, p_sigma=0.3)
    lam = np.random.default_rng(1).standard_normal((5,) + shape)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(n, k, to_gpu(lam, "f64"))
    dts = _oracle_dts(U0, shape, n)
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(lam), G, _dx(shape))
    assert _rel(g, ref) < 1e-10
    assert float((g.cpu() - ref).abs().max() / ref.abs().max()) < 1e-9


def test_kelvin_helmholtz_mass_invariant():
    """Piecewise-constant shear layer (on the limiter's kink almost everywhere): the gradient of
    the mean final density is exact on every branch."""
    shape = (16, 16, 16)
    U0 = inputs.kelvin_helmholtz(shape, seed=0)
    lam = np.zeros((5,) + shape)
    lam[0] = 1.0 / 16 ** 3
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(4, 2, to_gpu(lam, "f64")).cpu()
    assert float((g[0] - 1.0 / 16 ** 3).abs().max()) < 1e-15
    assert float(g[1:].abs().max()) < 1e-15


def test_central_finite_differences_fp64_16cubed():
    shape = (16, 16, 16)
    n = 10
    U0 = inputs.decaying_turbulence(shape, seed=2, sigma=0.5, mach=1.0, p_sigma=0.3)
    w = np.random.default_rng(3).standard_normal((5,) + shape)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(n, 3, to_gpu(w, "f64")).cpu()
    dts = _oracle_dts(U0, shape, n)
    wt = torch.from_numpy(w).cuda()

    def loss(U):
        f = solver(shape, "f64")
        f.init_state(to_gpu(U, "f64"))
        for dt in dts:
            f.step(dt, sync=False)
        return float((wt * f.get_state()).sum())

    rng = np.random.default_rng(4)
    for _ in range(8):
        i = tuple(int(rng.integers(0, d)) for d in (5,) + shape)
        eps = 1e-6 * max(1.0, abs(U0[i]))
        Up = U0.copy(); Up[i] += eps
        Um = U0.copy(); Um[i] -= eps
        fd = (loss(Up) - loss(Um)) / (2 * eps)
        assert fd == pytest.approx(float(g[i]), rel=1e-3, abs=1e-6), i


def test_dot_product_identity_fp64():
    shape = (12, 12, 12)
    n = 4
    U0 = inputs.decaying_turbulence(shape, seed=6, sigma=0.3, mach=0.6, p_sigma=0.3)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal((5,) + shape)
    v = rng.standard_normal((5,) + shape) * np.abs(U0).mean(axis=(1, 2, 3), keepdims=True)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    JTl = s.adjoint_advance(n, 2, to_gpu(lam, "f64")).cpu().numpy()
    dts = _oracle_dts(U0, shape, n)

    def fwd(U):
        f = solver(shape, "f64")
        f.init_state(to_gpu(U, "f64"))
        for dt in dts:
            f.step(dt, sync=False)
        return f.get_state().cpu().numpy()

    # a small step keeps the finite difference off the limiter's kinks (|a|, |b| ~ eps |U|)
    eps = 1e-8
    Jv = (fwd(U0 + eps * v) - fwd(U0 - eps * v)) / (2 * eps)
    a = float((lam * Jv).sum())
    b = float((JTl * v).sum())
    assert a == pytest.approx(b, rel=1e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mass_invariant(prec):
    shape = (16, 16, 16)
    U0 = inputs.decaying_turbulence(shape, seed=7, sigma=0.5, mach=1.5)
    N3 = 16 ** 3
    lam = np.zeros((5,) + shape)
    lam[0] = 1.0 / N3
    s = solver(shape, prec)
    s.init_state(to_gpu(U0, prec))
    g = s.adjoint_advance(8, 3, to_gpu(lam, prec)).double().cpu()
    tol = 1e-15 if prec == "f64" else 1e-9
    assert float((g[0] - 1.0 / N3).abs().max()) < tol
    assert float(g[1:].abs().max()) < tol


def test_fp32_matches_fp64_oracle_to_1e_3():
    shape = (32, 32, 32)
    n = 10
    U0 = inputs.decaying_turbulence(shape, seed=2, sigma=0.5, mach=2.0, p_sigma=0.3)
    lam = np.zeros((5,) + shape)
    rho_t = inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=2.0, p_sigma=0.3)[0]
    # MSE on the final density against a target (the reconstruction loss)
    dts = _oracle_dts(U0, shape, n)
    Uf = oadj.advance(torch.from_numpy(U0), dts, G, _dx(shape))
    lam[0] = 2.0 * (Uf[0].numpy() - rho_t) / rho_t.size
    s = solver(shape, "f32")
    s.init_state(to_gpu(U0, "f32"))
    g = s.adjoint_advance(n, 4, to_gpu(lam, "f32"))
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(lam), G, _dx(shape))
    assert _rel(g, ref) < 1e-3


def test_autograd_function_backward():
    from paper_2512_13403_b300 import autograd as dag
    shape = (16, 16, 16)
    U0 = to_gpu(inputs.decaying_turbulence(shape, seed=9, sigma=0.3, mach=0.7, p_sigma=0.3), "f64").requires_grad_(True)
    s = solver(shape, "f64")
    Un = dag.advance(U0, s, 5, 2)
    w = torch.randn_like(Un)
    (w * Un).sum().backward()
    s2 = solver(shape, "f64")
    s2.init_state(U0.detach())
    ref = s2.adjoint_advance(5, 5, w)
    assert torch.allclose(U0.grad, ref, rtol=1e-12, atol=1e-14)


def _gravity_case(shape, steps, forcing_cooling, seed=5):
    from oracle import driver
    U0 = inputs.decaying_turbulence(shape, seed=seed, sigma=0.5, mach=0.8, p_sigma=0.3)
    fc = dict(forcing=True, ou_seed=11, cooling=True, t_floor=0.05, cool_frac=0.02) if forcing_cooling else {}
    kw = dict(gravity=True, four_pi_G=1.0, mg_tol=1e-12, mg_max_cycles=60, **fc)
    cfg = driver.Config(shape=shape, gamma=G, **kw)
    sim = driver.Simulation(cfg, torch.from_numpy(U0))
    dts, fields = oadj.record(sim, steps)
    cool = dict(T_floor=0.05, frac=0.02, nsub_max=1024) if forcing_cooling else None
    return U0, dts, fields, cool, dict(four_pi_G=1.0), kw


@pytest.mark.parametrize("forcing_cooling", [False, True])
def test_fp64_with_gravity_matches_oracle(forcing_cooling):
    """Adjoint through self-gravity: the gravity kick transposed pointwise, then the potential's
    share through a second Poisson solve (the operator is symmetric)."""
    shape, n, k = (16, 16, 16), 4, 2
    U0, dts, fields, cool, grav, kw = _gravity_case(shape, n, forcing_cooling)
    lam = np.random.default_rng(5).standard_normal((5,) + shape)
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(n, k, to_gpu(lam, "f64"))
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(lam), G, _dx(shape),
                           fields if forcing_cooling else None, cool, grav)
    # the float64 context's multigrid runs float64 cycles: both Poisson solves are then exact to
    # far below the float64 bar of 1e-11 (measured: 1e-15)
    assert _rel(g, ref) < 1e-11
    assert float((g.cpu() - ref).abs().max() / ref.abs().max()) < 1e-11


def test_gravity_mass_invariant_fp32_and_state_kept():
    shape = (16, 16, 16)
    U0, dts, fields, cool, grav, kw = _gravity_case(shape, 4, True, seed=6)
    N3 = int(np.prod(shape))
    lam = np.zeros((5,) + shape)
    lam[0] = 1.0 / N3
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(4, 2, to_gpu(lam, "f64")).cpu()
    assert float((g[0] - 1.0 / N3).abs().max()) < 1e-14
    assert float(g[1:].abs().max()) < 1e-14
    # the context continues from the forward's final state and potential as if no adjoint ran
    s.advance(1)
    ref = solver(shape, "f64", **kw)
    ref.init_state(to_gpu(U0, "f64"))
    ref.advance(5)
    assert torch.equal(s.get_state().cpu(), ref.get_state().cpu())
    # float32 against the float64 oracle
    w = np.random.default_rng(8).standard_normal((5,) + shape)
    kw32 = dict(kw, mg_tol=1e-6, mg_max_cycles=30)
    s32 = solver(shape, "f32", **kw32)
    s32.init_state(to_gpu(U0, "f32"))
    g32 = s32.adjoint_advance(4, 2, to_gpu(w, "f32"))
    ref32 = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(w), G, _dx(shape), fields, cool, grav)
    assert _rel(g32, ref32) < 1e-3


def _source_case(shape, steps, seed=3):
    from oracle import driver
    U0 = inputs.decaying_turbulence(shape, seed=seed, sigma=0.5, mach=0.8, p_sigma=0.3)
    nz, ny, nx = shape
    cfg = driver.Config(shape=shape, gamma=G, forcing=True, ou_seed=11, cooling=True,
                        t_floor=0.05, cool_frac=0.02)
    sim = driver.Simulation(cfg, torch.from_numpy(U0))
    dts, fields = oadj.record(sim, steps)
    return U0, dts, fields, dict(T_floor=0.05, frac=0.02, nsub_max=1024)


@pytest.mark.parametrize("shape,n,k", [((16, 16, 16), 5, 2), ((12, 10, 20), 4, 4), ((8, 8, 64), 4, 2)])
def test_fp64_with_forcing_and_cooling_matches_oracle(shape, n, k):
    """Adjoint through RK2, the forcing kick (field of each step fixed) and subcycled cooling.
    On the 64-wide grid the forward sweep and the replayed segment run the paired stage kernel
    (with its staged forcing row factors and the pre-source capture)."""
    U0, dts, fields, cool = _source_case(shape, n)
    lam = np.random.default_rng(4).standard_normal((5,) + shape)
    s = solver(shape, "f64", forcing=True, ou_seed=11, cooling=True, t_floor=0.05, cool_frac=0.02)
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(n, k, to_gpu(lam, "f64"))
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(lam), G, _dx(shape), fields, cool)
    assert _rel(g, ref) < 1e-10
    assert float((g.cpu() - ref).abs().max() / ref.abs().max()) < 1e-9


def test_sources_mass_invariant_and_fp32():
    shape = (16, 16, 16)
    U0, dts, fields, cool = _source_case(shape, 4, seed=6)
    kw = dict(forcing=True, ou_seed=11, cooling=True, t_floor=0.05, cool_frac=0.02)
    N3 = int(np.prod(shape))
    lam = np.zeros((5,) + shape)
    lam[0] = 1.0 / N3
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(4, 2, to_gpu(lam, "f64")).cpu()
    assert float((g[0] - 1.0 / N3).abs().max()) < 1e-15
    assert float(g[1:].abs().max()) < 1e-15
    # float32 against the float64 oracle
    w = np.random.default_rng(7).standard_normal((5,) + shape)
    s32 = solver(shape, "f32", **kw)
    s32.init_state(to_gpu(U0, "f32"))
    g32 = s32.adjoint_advance(4, 2, to_gpu(w, "f32"))
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(w), G, _dx(shape), fields, cool)
    assert _rel(g32, ref) < 1e-3


SCHEMES = [("rk2", "vanleer"), ("ssprk3", "mc"), ("ssprk3", "vanleer")]


@pytest.mark.parametrize("integrator,limiter", SCHEMES)
def test_scheme_variants_match_oracle_vjp(integrator, limiter):
    """Hand adjoint of SSPRK3 and of the van Leer slope against reverse mode of the oracle."""
    shape, n, k = (12, 10, 20), 4, 3
    U0 = inputs.decaying_turbulence(shape, seed=5, sigma=0.3, mach=0.8, p_sigma=0.3)
    lam = np.random.default_rng(1).standard_normal((5,) + shape)
    s = solver(shape, "f64", integrator=integrator, limiter=limiter)
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(n, k, to_gpu(lam, "f64"))
    scheme = dict(integrator=integrator, limiter=limiter)
    U = torch.from_numpy(U0)
    dts = []
    for _ in range(n):
        dts.append(ohydro.cfl_dt(U, G, _dx(shape), 0.4))
        U = ohydro.step(U, dts[-1], G, _dx(shape), integrator, limiter)
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(lam), G, _dx(shape),
                           scheme=scheme)
    assert _rel(g, ref) < 1e-10
    assert float((g.cpu() - ref).abs().max() / ref.abs().max()) < 1e-9


@pytest.mark.parametrize("integrator,limiter", [("ssprk3", "vanleer")])
def test_scheme_variant_with_sources_matches_oracle_vjp(integrator, limiter):
    shape, n, k = (16, 16, 16), 4, 2
    from oracle import driver
    U0 = inputs.decaying_turbulence(shape, seed=8, sigma=0.4, mach=0.6, P0=0.6, p_sigma=0.3)
    kw = dict(forcing=True, ou_seed=11, cooling=True, t_floor=0.05, cool_frac=0.02,
              integrator=integrator, limiter=limiter)
    sim = driver.Simulation(driver.Config(shape=shape, gamma=G, **kw), torch.from_numpy(U0))
    dts, fields = oadj.record(sim, n)
    lam = np.random.default_rng(4).standard_normal((5,) + shape)
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    g = s.adjoint_advance(n, k, to_gpu(lam, "f64"))
    ref = oadj.advance_vjp(torch.from_numpy(U0), dts, torch.from_numpy(lam), G, _dx(shape), fields,
                           dict(T_floor=0.05, frac=0.02, nsub_max=1024),
                           scheme=dict(integrator=integrator, limiter=limiter))
    assert _rel(g, ref) < 1e-10


@pytest.mark.parametrize("prec,integrator,sources", [("f32", "rk2", False), ("f32", "ssprk3", True),
                                                     ("f64", "rk2", True)])
def test_gradient_independent_of_checkpoint_interval(prec, integrator, sources):
    """The states of a segment are recomputed bit for bit, and the last segment's are kept from
    the forward sweep instead, so the gradient is the same bits for every checkpoint interval
    (one segment held whole, several replayed, one step per segment)."""
    shape = (12, 10, 20)
    n = 7
    U0 = inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=0.8, p_sigma=0.3)
    kw = dict(forcing=True, ou_seed=5, cooling=True, t_floor=0.05, cool_frac=0.02) if sources else {}
    lam = to_gpu(np.random.default_rng(8).standard_normal((5,) + shape), prec)
    grads = []
    for k in (n, 3, 1):
        s = solver(shape, prec, integrator=integrator, **kw)
        s.init_state(to_gpu(U0, prec))
        grads.append(s.adjoint_advance(n, k, lam).clone())
        s.close()
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_adjoint_commutes_with_reflection_fp64(axis):
    """The gradient of the reflected problem (state and lambda reflected, the momentum along the
    axis negated in both) is the reflected gradient."""
    shape = (12, 10, 20)
    U0 = torch.from_numpy(inputs.decaying_turbulence(shape, seed=5, sigma=0.3, mach=0.8, p_sigma=0.3))
    lam = torch.from_numpy(np.random.default_rng(3).standard_normal((5,) + shape))

    def mirror(U):
        d = 3 - axis
        V = torch.flip(U, dims=[d]).clone()
        V[1 + axis] = -V[1 + axis]
        return V

    grads = []
    for U, L in ((U0, lam), (mirror(U0), mirror(lam))):
        s = solver(shape, "f64")
        s.init_state(to_gpu(U.numpy(), "f64"))
        grads.append(s.adjoint_advance(3, 2, to_gpu(L.numpy(), "f64")).cpu())
        s.close()
    assert _rel(mirror(grads[1]), grads[0]) < 1e-11


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_translation_equivariant(prec):
    """The gradient of a periodically shifted problem is the shifted gradient: bit for bit for
    shifts in x and y, to rounding for shifts in z (z-chunk starts take their first faces and
    slope terms from the prologue's copy of the same formulas)."""
    shape = (12, 10, 20)
    U0 = torch.from_numpy(inputs.decaying_turbulence(shape, seed=5, sigma=0.3, mach=0.8, p_sigma=0.3))
    lam = torch.from_numpy(np.random.default_rng(3).standard_normal((5,) + shape))

    def grad(U, L):
        s = solver(shape, prec)
        s.init_state(to_gpu(U.numpy(), prec))
        g = s.adjoint_advance(3, 2, to_gpu(L.numpy(), prec)).cpu()
        s.close()
        return g

    ref = grad(U0, lam)
    for shift, exact in (((0, 3, 11), True), ((5, 3, 11), False)):
        got = grad(torch.roll(U0, shift, (1, 2, 3)), torch.roll(lam, shift, (1, 2, 3)))
        want = torch.roll(ref, shift, (1, 2, 3))
        if exact:
            assert torch.equal(want, got), shift
        else:
            assert _rel(got, want) < (1e-13 if prec == "f64" else 1e-5), shift


def test_adjoint_edge_cases():
    """n = 0 returns lambda unchanged; a checkpoint interval larger than n is one kept segment
    (same bits as k = n); bad arguments are rejected without touching the state."""
    from paper_2512_13403_b300._lib import DH_ERR_ARG, DhError
    shape = (8, 8, 8)
    U0 = inputs.decaying_turbulence(shape, seed=2, sigma=0.3, mach=0.6, p_sigma=0.2)
    lam = to_gpu(np.random.default_rng(2).standard_normal((5,) + shape), "f64")
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    assert torch.equal(s.adjoint_advance(0, 1, lam), lam)
    g_big = s.adjoint_advance(3, 50, lam).clone()
    s.init_state(to_gpu(U0, "f64"))
    assert torch.equal(s.adjoint_advance(3, 3, lam), g_big)
    t0 = s.time()
    for n, k in ((-1, 1), (2, 0)):
        with pytest.raises(DhError) as e:
            s.adjoint_advance(n, k, lam)
        assert e.value.status == DH_ERR_ARG
    assert s.time() == t0
    s.close()
