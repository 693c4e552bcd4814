"""GPU parity of the paired stage kernel (grids of whole 64 x 8 tiles; hydro_pair.cu) through the
C ABI against the FP64 CPU oracle: the two cells of a thread sit 32 apart in x, planes arrive by
tensor-map boxes, and the update of each plane runs one plane behind its fluxes."""
import numpy as np
import pytest
import torch

from oracle import driver as odrv
from oracle import hydro as ohydro
from paper_2512_13403_b300 import inputs
from tests.gpu_util import rel_l1, rel_linf, solver, to_gpu

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0
SCHEMES = [("ssprk3", "mc"), ("rk2", "vanleer"), ("ssprk3", "vanleer")]


def _dx(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


# (nz, ny, nx): one tile with both halos wrapping onto itself; several z chunks of one tile;
# two x tiles with a 5-plane box; the smallest z extent the kernel takes; several y tiles
SHAPES = [(12, 16, 64), (40, 8, 64), (5, 8, 128), (4, 16, 64), (10, 24, 64)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_paired_tiles_with_sources(shape, prec, tol):
    """Three steps with OU forcing and cooling against the oracle (float64 with its own CFL
    steps, float32 on the oracle's time steps)."""
    U0 = inputs.decaying_turbulence(shape, seed=7, sigma=0.4, mach=1.0, p_sigma=0.2)
    kw = dict(forcing=min(shape) >= 5, cooling=True)   # the forcing modes need 5 cells per axis
    sim = odrv.Simulation(odrv.Config(shape=shape, **kw), U0)
    s = solver(shape, prec, **kw)
    s.init_state(to_gpu(U0, prec))
    for _ in range(3):
        if prec == "f64":
            dt = s.step(0.0)
            assert dt == pytest.approx(sim.compute_dt(), rel=1e-13)
        else:
            dt = s.step(sim.compute_dt())
        sim.step(dt)
    assert max(rel_linf(s.get_state(), sim.U)) <= tol


def test_paired_kh_fp64_and_fp32():
    """The Kelvin-Helmholtz shear layer (configuration 1's initial state) on a 64-wide box, ten
    steps: float64 to 1e-11, float32 to 1e-5 relative L1 per field."""
    shape = (16, 32, 64)
    U0 = inputs.kelvin_helmholtz(shape, seed=0)
    sim = odrv.Simulation(odrv.Config(shape=shape), U0)
    dts = sim.advance(10)
    s64 = solver(shape, "f64")
    s64.init_state(to_gpu(U0, "f64"))
    s64.advance(10)
    assert max(rel_linf(s64.get_state(), sim.U, own_scale=True)) <= 1e-11
    s32 = solver(shape, "f32")
    s32.init_state(to_gpu(U0, "f32"))
    for dt in dts:
        s32.step(dt, sync=False)
    e = rel_l1(s32.get_state(), sim.U)
    assert max(e[i] for i in (0, 1, 4)) <= 1e-5, e


@pytest.mark.parametrize("integrator,limiter", SCHEMES)
def test_paired_scheme_variants_fp64(integrator, limiter):
    """Van Leer and SSPRK3 (App. A.1, A.3) in the paired kernel, three CFL steps."""
    shape = (16, 8, 64)
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


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paired_translation_equivariant(prec):
    """A periodically shifted state steps to the shifted result bit for bit: shifts in x that
    move cells between the two lanes of a thread (32), across a lane's halo (1, 31, 33) and
    across tiles (64); shifts in y across rows and tiles; shifts in z across z-chunk starts."""
    shape = (24, 16, 128)
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
    for shift in ((0, 0, 1), (0, 0, 31), (0, 0, 32), (0, 0, 33), (0, 0, 64), (0, 3, 0), (0, 8, 0),
                  (7, 0, 0), (13, 5, 37)):
        got = run(torch.roll(U0, shifts=shift, dims=(1, 2, 3)))
        want = torch.roll(ref, shifts=shift, dims=(1, 2, 3))
        assert torch.equal(want, got), shift


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paired_fallback_count(prec):
    """The positivity-fallback count of the paired kernel: density repeats (tiny, 1, 4) along x
    at rest, so the middle cell of each triple falls back on the x axis in both RK stages and no
    other cell or axis does (2 nz ny nx / 3 events per step)."""
    nz, ny, nx = 6, 8, 192
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


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paired_cfl_minimum_equals_cfl_reduce(prec):
    """The CFL minimum that the paired kernel's final stage reduces (and the next step takes as
    its dt) is bit for bit the one cfl_reduce_kernel computes from the same state: a step taken
    after one step equals the CFL step recomputed on that state in a second context."""
    shape = (12, 16, 64)
    U0 = inputs.decaying_turbulence(shape, seed=8, sigma=0.5, mach=1.2, p_sigma=0.3)
    kw = dict(forcing=True, cooling=True)
    a = solver(shape, prec, **kw)
    b = solver(shape, prec, **kw)
    a.init_state(to_gpu(U0, prec))
    b.init_state(to_gpu(U0, prec))
    assert a.step(0.0) == b.step(0.0)
    dt2 = a.step(0.0)               # from the first step's fused CFL reduction
    assert b.compute_dt() == dt2    # recomputed by the stand-alone reduction on the same state
