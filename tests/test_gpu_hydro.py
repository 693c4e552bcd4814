"""GPU parity of the hydro step through the C ABI against the FP64 CPU oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import cooling as ocool
from oracle import driver as odrv
from oracle import forcing as oforce
from oracle import hydro as ohydro
from paper_2512_13403_b300 import inputs
from tests.gpu_util import rel_l1, rel_l1_vector_scaled, rel_linf, solver, to_gpu

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _dx(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


def test_single_step_fp64_kh32():
    shape = (32, 32, 32)
    U0 = inputs.kelvin_helmholtz(shape, seed=0)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    dt = ohydro.cfl_dt(torch.from_numpy(U0), G, _dx(shape), 0.4)
    s.step(dt)
    ref = ohydro.rk2_step(torch.from_numpy(U0), dt, G, _dx(shape))
    assert max(rel_linf(s.get_state(), ref)) <= 1e-11


@pytest.mark.parametrize("shape", [(12, 16, 64), (8, 8, 32), (6, 24, 96)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_tensor_map_tiles_with_sources(shape, prec, tol):
    """Grids of whole 32 x 8 tiles, whose planes arrive by tensor-map (TMA) boxes: the tile core
    and four halo strips, each wrapped to the other side of the periodic box at the edges; with
    one tile across an axis both of its halos wrap onto the tile itself.  Three steps with
    forcing and cooling against the oracle."""
    U0 = inputs.decaying_turbulence(shape, seed=7, sigma=0.4, mach=1.0, p_sigma=0.2)
    kw = dict(forcing=True, cooling=True)
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, prec, **kw)
    s.init_state(to_gpu(U0, prec))
    for _ in range(3):
        dt = s.step(0.0 if prec == "f64" else sim.compute_dt())
        sim.step(dt)
    assert max(rel_linf(s.get_state(), sim.U)) <= tol


@pytest.mark.parametrize("shape", [(20, 12, 40), (9, 17, 33), (8, 8, 70)])
def test_ragged_tiles_fp64(shape):
    U0 = inputs.decaying_turbulence(shape, seed=3, sigma=0.4, mach=1.0)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    U = torch.from_numpy(U0)
    for _ in range(3):
        dt = s.step(0.0)
        dto = ohydro.cfl_dt(U, G, _dx(shape), 0.4)
        assert dt == pytest.approx(dto, rel=1e-13)
        U = ohydro.rk2_step(U, dto, G, _dx(shape))
    assert max(rel_linf(s.get_state(), U)) <= 1e-11


@pytest.mark.parametrize("shape", [(4, 6, 5), (5, 4, 8), (6, 5, 4)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_smallest_grids(shape, prec, tol):
    """Grids of 4-8 cells per axis: every staged plane, halo row and face wraps around the
    periodic box, and rows of 5 or 4 cells take the element or 16-byte staging copies."""
    U0 = inputs.decaying_turbulence(shape, seed=4, sigma=0.4, mach=1.0)
    s = solver(shape, prec)
    s.init_state(to_gpu(U0, prec))
    U = torch.from_numpy(to_gpu(U0, prec).double().cpu().numpy())
    for _ in range(3):
        dto = ohydro.cfl_dt(U, G, _dx(shape), 0.4)
        s.step(dto)
        U = ohydro.rk2_step(U, dto, G, _dx(shape))
    assert max(rel_linf(s.get_state(), U)) <= tol


def test_kh32_50_steps_fp64_and_fp32():
    shape = (32, 32, 32)
    U0 = inputs.kelvin_helmholtz(shape, seed=0)
    sim = odrv.Simulation(odrv.Config(shape=shape), U0)
    dts = sim.advance(50)
    ref = sim.U
    s64 = solver(shape, "f64")
    s64.init_state(to_gpu(U0, "f64"))
    t64 = s64.advance(50)
    assert t64 == pytest.approx(sim.t, rel=1e-12)
    assert max(rel_linf(s64.get_state(), ref, own_scale=True)) <= 1e-11
    # FP32 production path: dt schedule replayed, then self-computed dt.  The shear layer is a
    # discontinuous flow whose transverse momenta are 1% perturbations of the O(1) shear, so
    # momentum components are measured against the momentum-magnitude scale.
    s32 = solver(shape, "f32")
    s32.init_state(to_gpu(U0, "f32"))
    for dt in dts:
        s32.step(dt, sync=False)
    e = rel_l1_vector_scaled(s32.get_state(), ref)
    assert max(e) <= 1e-5, e
    assert max(rel_l1(s32.get_state(), ref)[i] for i in (0, 1, 4)) <= 1e-5
    s32b = solver(shape, "f32")
    s32b.init_state(to_gpu(U0, "f32"))
    s32b.advance(50)
    e = rel_l1_vector_scaled(s32b.get_state(), ref)
    assert max(e) <= 1e-5, e


def test_smooth_flow_50_steps_fp32_every_field():
    """FP32 vs oracle on a smooth flow: 1e-5 relative L1 on every field, each on its own scale."""
    shape = (32, 32, 32)
    U0 = inputs.decaying_turbulence(shape, seed=2, sigma=0.3, mach=0.5)
    sim = odrv.Simulation(odrv.Config(shape=shape), U0)
    dts = sim.advance(50)
    s32 = solver(shape, "f32")
    s32.init_state(to_gpu(U0, "f32"))
    for dt in dts:
        s32.step(dt, sync=False)
    e = rel_l1(s32.get_state(), sim.U)
    assert max(e) <= 1e-5, e


def test_ou_table_over_many_steps_and_a_rollback():
    """The OU draws of many steps are made ahead of the steps in batches of 128; the mode table
    after 300 fixed-dt steps (three batches, plus a reload that rewinds the step count) is the
    oracle's OU recurrence to rounding."""
    from paper_2512_13403_b300 import _lib
    shape = (8, 8, 8)
    U0 = inputs.decaying_turbulence(shape, seed=2, sigma=0.3, mach=0.2, P0=1.0)
    s = solver(shape, "f64", forcing=True, ou_tau=0.5, ou_arms=0.1, ou_seed=5)
    s.init_state(to_gpu(U0, "f64"))
    ou = oforce.OUForcing(5, 0.5, 0.1)
    dt = 1e-3
    for n in range(1, 301):
        s.step(dt, sync=False)
        ou.update(dt, n - 1)   # step n (1-based) takes draw n
        if n == 150:
            assert np.abs(s.forcing_modes() - ou.a_hat.numpy()).max() < 1e-12
    assert np.abs(s.forcing_modes() - ou.a_hat.numpy()).max() < 1e-12
    # a step count rewound by a reload: the next steps draw from the right place again
    import os, tempfile
    path = os.path.join(tempfile.mkdtemp(), "ck.bin")
    s2 = solver(shape, "f64", forcing=True, ou_tau=0.5, ou_arms=0.1, ou_seed=5)
    s2.init_state(to_gpu(U0, "f64"))
    ou2 = oforce.OUForcing(5, 0.5, 0.1)
    for n in range(1, 11):
        s2.step(dt)
        ou2.update(dt, n - 1)
    s2.save(path)
    for n in range(11, 141):
        s2.step(dt, sync=False)
    s2.load(path)
    for n in range(11, 21):
        s2.step(dt)
        ou2.update(dt, n - 1)
    assert np.abs(s2.forcing_modes() - ou2.a_hat.numpy()).max() < 1e-12


def test_forcing_and_cooling_fp64():
    shape = (16, 20, 24)
    U0 = inputs.decaying_turbulence(shape, seed=9, sigma=0.5, mach=0.7, P0=0.6)
    kw = dict(forcing=True, ou_tau=0.5, ou_arms=1.0, ou_seed=1, cooling=True, t_floor=0.05)
    sim = odrv.Simulation(odrv.Config(shape=shape, forcing=True, cooling=True, ou_seed=1), U0)
    s = solver(shape, "f64", **kw)
    s.init_state(to_gpu(U0, "f64"))
    # initial mode table: draw 0 of the counter-based stream, projected
    assert np.abs(s.forcing_modes() - sim.ou.a_hat.numpy()).max() < 1e-14
    for _ in range(4):
        dt = s.step(0.0)
        dto = sim.step()
        assert dt == pytest.approx(dto, rel=1e-13)
    assert np.abs(s.forcing_modes() - sim.ou.a_hat.numpy()).max() < 1e-13
    a = s.forcing_field()
    assert max(rel_linf(a, sim.ou.field(shape))) < 1e-12
    assert max(rel_linf(s.get_state(), sim.U)) <= 1e-11


def test_cooling_subcycling_branch_fp64():
    """Dense hot cells force N_sub > 1; compare against the oracle's subcycled update."""
    shape = (8, 8, 8)
    rng = np.random.default_rng(4)
    rho = np.exp(rng.normal(0, 1.0, shape)) * 5.0
    P = np.full(shape, 3.0)
    z = np.zeros(shape)
    U0 = inputs.prim_to_state(rho, z + 0.1, z, z, P, G)
    sim = odrv.Simulation(odrv.Config(shape=shape, cooling=True, t_floor=0.05), U0)
    s = solver(shape, "f64", cooling=True, t_floor=0.05)
    s.init_state(to_gpu(U0, "f64"))
    dt = 0.01
    nsub, _ = ocool.substep_count(torch.from_numpy(U0[4] - 0.5 * U0[1] ** 2 / U0[0]),
                                  torch.from_numpy(U0[0]), dt, G, 0.05)
    assert float(nsub.max()) > 1.0  # the subcycled branch is exercised
    s.step(dt)
    sim.step(dt)
    assert max(rel_linf(s.get_state(), sim.U)) <= 1e-11


@pytest.mark.parametrize("shape", [(12, 16, 20), (9, 11, 13), (33, 17, 35)])
def test_conserved_totals_fp64_and_fp32(shape):
    """Totals against math.fsum; cell counts that are multiples of 4 take the float32 path's
    16-byte loads, odd ones its element loads."""
    U0 = inputs.kelvin_helmholtz(shape, seed=1)
    for prec in ("f64", "f32"):
        s = solver(shape, prec)
        Ug = to_gpu(U0, prec)
        s.init_state(Ug)
        tot = s.conserved_totals()
        exact = [math.fsum(Ug[f].double().cpu().reshape(-1).tolist()) for f in range(5)]
        for f in range(5):
            assert tot[f] == pytest.approx(exact[f], rel=1e-13, abs=1e-12)
        s.advance(5)
        tot2 = s.conserved_totals()
        tol = 1e-12 if prec == "f64" else 2e-6
        for f in (0, 4):
            assert abs(tot2[f] - tot[f]) <= tol * abs(tot[f])


def test_argument_and_state_errors():
    from paper_2512_13403_b300._lib import DH_ERR_ARG, DH_ERR_STATE, DhError
    with pytest.raises(DhError) as e:
        solver((2, 8, 8), "f64")
    assert e.value.status == DH_ERR_ARG
    with pytest.raises(DhError) as e:
        solver((8, 8, 8), "f64", forcing=True, ou_tau=-1.0)
    assert e.value.status == DH_ERR_ARG
    s = solver((8, 8, 8), "f64")
    with pytest.raises(DhError) as e:
        s.step(0.0)
    assert e.value.status == DH_ERR_STATE


def test_nonfinite_and_positivity_keep_last_good_state():
    from paper_2512_13403_b300._lib import DH_ERR_NONFINITE, DH_ERR_POSITIVITY, DhError
    shape = (8, 8, 16)
    U0 = inputs.decaying_turbulence(shape, seed=1, sigma=0.3, mach=0.5)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    s.advance(2)
    good = s.get_state().clone()
    t_good, n_good = s.time()
    # host-side fault injection: a NaN in the uploaded state
    bad = good.clone()
    bad[4, 3, 3, 3] = float("nan")
    s.init_state(bad)
    with pytest.raises(DhError) as e:
        s.step(1e-4)
    assert e.value.status == DH_ERR_NONFINITE
    assert torch.equal(s.get_state().isnan(), bad.isnan())
    assert s.time() == (0.0, 0)
    # negative pressure after a step: a huge dt on a strong rarefaction
    s.init_state(good)
    s.step(1e-4)
    kept = s.get_state().clone()
    with pytest.raises(DhError) as e:
        s.step(10.0)
    assert e.value.status in (DH_ERR_POSITIVITY, DH_ERR_NONFINITE)
    assert torch.equal(s.get_state(), kept)
    t, n = s.time()
    assert n == 1 and t == pytest.approx(1e-4)
    # the context stays usable
    s.advance(2)


def test_cfl_dt_matches_oracle():
    shape = (10, 12, 14)
    U0 = inputs.decaying_turbulence(shape, seed=8, mach=2.0)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    assert s.compute_dt() == pytest.approx(ohydro.cfl_dt(torch.from_numpy(U0), G, _dx(shape), 0.4),
                                           rel=1e-14)


SCHEMES = [("rk2", "vanleer"), ("ssprk3", "mc"), ("ssprk3", "vanleer")]


@pytest.mark.parametrize("integrator,limiter", SCHEMES)
@pytest.mark.parametrize("shape", [(16, 16, 16), (9, 17, 33)])
def test_scheme_variants_fp64(shape, integrator, limiter):
    """Van Leer limiter and SSPRK3 (App. A.1, A.3) against the oracle, three CFL steps."""
    U0 = inputs.decaying_turbulence(shape, seed=3, sigma=0.4, mach=1.0)
    s = solver(shape, "f64", integrator=integrator, limiter=limiter)
    s.init_state(to_gpu(U0, "f64"))
    U = torch.from_numpy(U0)
    for _ in range(3):
        dt = s.step(0.0)
        dto = ohydro.cfl_dt(U, G, _dx(shape), 0.4)
        assert dt == pytest.approx(dto, rel=1e-13)
        U = ohydro.step(U, dto, G, _dx(shape), integrator, limiter)
    assert max(rel_linf(s.get_state(), U)) <= 1e-11


@pytest.mark.parametrize("integrator,limiter", SCHEMES)
def test_scheme_variants_with_sources_fp64_and_fp32(integrator, limiter):
    shape = (16, 20, 24)
    U0 = inputs.decaying_turbulence(shape, seed=9, sigma=0.5, mach=0.7, P0=0.6)
    kw = dict(forcing=True, ou_seed=1, cooling=True, t_floor=0.05, integrator=integrator,
              limiter=limiter)
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, "f64", **kw)
    s32 = solver(shape, "f32", **kw)
    s.init_state(to_gpu(U0, "f64"))
    s32.init_state(to_gpu(U0, "f32"))
    for _ in range(4):
        dt = s.step(0.0)
        s32.step(dt)
        dto = sim.step()
        assert dt == pytest.approx(dto, rel=1e-13)
    assert max(rel_linf(s.get_state(), sim.U)) <= 1e-11
    assert max(rel_linf(s32.get_state(), sim.U)) <= 1e-5


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_cooling_time_step_limit(prec, tol):
    """dt = min(CFL step, c_cool min t_cool, dt_max) (Sec. 4.3), reduced in the stage-2 epilogue
    (and after init_state) on the GPU, against the oracle's step; the limit binds here."""
    shape = (16, 20, 24)
    U0 = inputs.decaying_turbulence(shape, seed=9, sigma=0.5, mach=0.7, P0=0.6)
    kw = dict(forcing=True, ou_seed=1, cooling=True, t_floor=0.05, c_cool=0.01)
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), to_gpu(U0, prec).double().cpu())
    s = solver(shape, prec, **kw)
    s.init_state(to_gpu(U0, prec))
    for _ in range(4):
        cfl = ohydro.cfl_dt(sim.U, G, _dx(shape), 0.4)
        dto = sim.step()
        assert dto < 0.9 * cfl
        dt = s.step(0.0)
        assert dt == pytest.approx(dto, rel=1e-13 if prec == "f64" else 2e-6)
    assert max(rel_linf(s.get_state(), sim.U)) <= tol


def _mirror(U, axis):
    """Reflection x_a -> -x_a of a periodic cell-centred state (fields, z, y, x): cell i goes to
    n - 1 - i and the momentum along the axis changes sign."""
    d = 3 - axis
    V = torch.flip(U, dims=[d]).clone()
    V[1 + axis] = -V[1 + axis]
    return V


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_step_commutes_with_reflection(axis, prec, tol):
    """The scheme treats both directions of an axis alike (MC, HLLC and the divergence are
    mirror-symmetric), so a step of the reflected state is the reflected step, up to the
    rounding of the differently ordered operations; a halo or face-index slip on either side of
    a tile would break it.  Ragged tiles in x and y, several z chunks."""
    shape = (20, 12, 40)
    U0 = torch.from_numpy(inputs.decaying_turbulence(shape, seed=8, sigma=0.5, mach=1.2))
    dt = 0.8 * ohydro.cfl_dt(U0, G, _dx(shape), 0.4)
    out = []
    for U in (U0, _mirror(U0, axis)):
        s = solver(shape, prec)
        s.init_state(to_gpu(U, prec))
        s.step(dt)
        out.append(s.get_state().cpu())
        s.close()
    assert max(rel_linf(_mirror(out[1], axis), out[0])) <= tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_step_translation_equivariant(prec):
    """A periodically shifted state steps to the shifted result (cooling on; the forcing field
    is position-dependent and is off here), bit for bit in every axis: every cell's update is
    the same code wherever it sits in its tile, staging chunk or z chunk.  Shifts in z move cells
    across z-chunk starts, whose first z face and slope the prologue evaluates; the formulas
    round alike there because their products and sums are spelled out with fixed rounding."""
    shape = (20, 12, 40)
    U0 = torch.from_numpy(inputs.decaying_turbulence(shape, seed=6, sigma=0.5, mach=1.2))

    def run(U):
        s = solver(shape, prec, cooling=True, t_floor=0.05)
        s.init_state(to_gpu(U, prec))
        for _ in range(2):
            s.step(0.0)
        out = s.get_state().cpu()
        s.close()
        return out

    ref = run(U0)
    for shift in ((0, 5, 13), (7, 5, 13), (1, 0, 0)):
        got = run(torch.roll(U0, shifts=shift, dims=(1, 2, 3)))
        want = torch.roll(ref, shifts=shift, dims=(1, 2, 3))
        assert torch.equal(want, got), shift


def test_metrics_record_cooling_cap_and_minima():
    """dh_get_metrics: a step whose cooling needs more substeps than nsub_max raises
    DH_FLAG_COOL_CAP and reports nsub_max as the largest substep count; the totals equal
    dh_conserved_totals, the minima those of the state, and the substep maximum covers the
    interval since the previous read."""
    from paper_2512_13403_b300 import _lib
    shape = (16, 16, 16)
    U0 = inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=0.5)
    # strong cooling: a large density contrast and a small substep cap
    s = solver(shape, "f64", cooling=True, t_floor=0.01, cool_frac=0.01, nsub_max=4)
    s.init_state(to_gpu(U0, "f64"))
    m0 = s.metrics()
    assert m0["nstep"] == 0 and m0["cool_max_substeps"] == 0 and m0["flags"] == 0
    s.step(0.0)
    m = s.metrics()
    assert m["nstep"] == 1 and m["dt"] > 0
    assert m["flags"] & _lib.DH_FLAG_COOL_CAP
    assert m["cool_max_substeps"] == 4
    assert m["totals"] == pytest.approx(s.conserved_totals(), rel=1e-14)
    U = s.get_state().cpu()
    P = (5.0 / 3.0 - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
    assert m["rho_min"] == float(U[0].min())
    assert m["p_min"] == pytest.approx(float(P.min()), rel=1e-12)
    assert m["mg_cycles"] == 0
    # the read reset the interval maximum: with no step since, cooling reports no subcycling
    assert s.metrics()["cool_max_substeps"] == 1
    assert m["slope_fallbacks"] == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_metrics_count_slope_fallbacks(prec):
    """The positivity fallback of the PLM slopes (App. A.2) is counted once per (cell, axis,
    RK stage).  Density repeats (tiny, 1, 4) along x at rest under uniform pressure: the middle
    cell's MC slope is 2 (the limit 2|b| with b = 1 - tiny, which rounds to 1), so its lower face
    density 1 - 2/2 is exactly 0 and the fallback fires on the x axis; no other cell or axis
    can fire (the slopes of the outer cells change sign, y and z are uniform).  A fixed time
    step far below the rounding of the state leaves U1 = U^n, so both stages fire alike:
    2 nz ny nx / 3 events per step.  x = 48 is not a multiple of the staging tile, so a partial
    tile is covered as well."""
    nz, ny, nx = 6, 10, 48
    tiny = 1e-20 if prec == "f64" else 1e-9
    U = np.zeros((5, nz, ny, nx))
    U[0] = np.tile(np.array([tiny, 1.0, 4.0]), nx // 3)[None, None, :]
    U[4] = 1.0 / (5.0 / 3.0 - 1.0)
    s = solver((nz, ny, nx), prec)
    s.init_state(to_gpu(U, prec))
    s.step(1e-30)
    m = s.metrics()
    assert m["flags"] == 0
    assert m["slope_fallbacks"] == 2 * nz * ny * nx // 3
    s.step(1e-30)
    s.step(1e-30)
    assert s.metrics()["slope_fallbacks"] == 4 * nz * ny * nx // 3
    assert s.metrics()["slope_fallbacks"] == 0
    # a smooth state with positive neighbours never falls back
    s2 = solver((8, 8, 32), prec)
    s2.init_state(to_gpu(inputs.decaying_turbulence((8, 8, 32), seed=5, sigma=0.5, mach=0.5), prec))
    for _ in range(3):
        s2.step(0.0)
    assert s2.metrics()["slope_fallbacks"] == 0
