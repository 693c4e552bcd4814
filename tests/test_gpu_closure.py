"""The closure workflow's library pieces on the GPU: 4^3 block mean, held forcing tables, the
context corrector, and a small end-to-end pair/train/evaluate cycle."""
import numpy as np
import pytest
import torch

from oracle import corrector as oc
from paper_2512_13403_b300 import closure, inputs
from paper_2512_13403_b300.corrector import NPARAM, init_params, unflatten
from tests.gpu_util import solver, to_gpu

pytestmark = pytest.mark.gpu


def test_downsample_is_block_mean():
    U = torch.rand(5, 16, 24, 32, dtype=torch.float32, device="cuda")
    D = closure.downsample(U, 4)
    ref = U.double().reshape(5, 4, 4, 6, 4, 8, 4).mean(dim=(2, 4, 6))
    assert torch.allclose(D.double(), ref, rtol=1e-6, atol=1e-7)


def test_held_forcing_table_is_kept():
    shape = (16, 16, 16)
    s = solver(shape, "f32", forcing=True)
    s.init_state(to_gpu(inputs.cooling_box(shape), "f32"))
    rng = np.random.default_rng(0)
    modes = rng.standard_normal((16, 3)) + 1j * rng.standard_normal((16, 3))
    s.set_forcing_modes(modes, hold=True)
    s.advance(3)
    assert np.array_equal(s.forcing_modes(), modes)
    s.set_forcing_modes(modes, hold=False)
    s.advance(1)
    assert not np.array_equal(s.forcing_modes(), modes)


def test_context_corrector_matches_oracle_and_zero_is_identity():
    import ctypes as C
    from paper_2512_13403_b300 import _lib
    shape = (8, 16, 16)
    U0 = inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=1.0, p_sigma=0.2)
    s = solver(shape, "f32")
    s.init_state(to_gpu(U0, "f32"))
    lib = _lib.load()
    with pytest.raises(_lib.DhError):
        _lib.check(lib.dh_correct(s.ctx), s.ctx)
    mu = [float(U0[c].mean()) for c in range(5)]
    sg = [float(U0[c].std()) for c in range(5)]
    out = [0.01 * v for v in sg]
    p = init_params(1, out_scale=1.0).cuda()
    norm = (C.c_float * 15)(*(mu + sg + out))
    _lib.check(lib.dh_set_corrector(s.ctx, C.c_void_p(p.data_ptr()), norm), s.ctx)
    _lib.check(lib.dh_correct(s.ctx), s.ctx)
    got = s.get_state().double().cpu()
    Uf = torch.from_numpy(U0).float().double()
    ref = oc.correct(Uf, unflatten(p.double().cpu()), mu, sg, 1e-6 * float(Uf[0].mean()), 0.05, 5 / 3,
                     out_scale=out)
    # the corrections agree to the BF16 activation rounding; the state itself to float32
    assert float((got - ref).abs().max() / (ref - Uf).abs().max()) < 2e-2
    # zero network: identity
    s.init_state(to_gpu(U0, "f32"))
    z = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
    _lib.check(lib.dh_set_corrector(s.ctx, C.c_void_p(z.data_ptr()), norm), s.ctx)
    _lib.check(lib.dh_correct(s.ctx), s.ctx)
    assert torch.equal(s.get_state().cpu(), torch.from_numpy(U0).float())


def test_small_pair_train_evaluate_cycle():
    setup = closure.ClosureSetup(fine=32, factor=4, runs=2, snapshots=6, spinup_steps=10)
    X, Y = closure.make_pairs(setup)
    assert X.shape == (12, 5, 8, 8, 8) and torch.isfinite(X).all() and torch.isfinite(Y).all()
    # the coarse step and the downsampled fine run differ, but not by much
    rel = float((Y - X).norm() / Y.norm())
    assert 0.0 < rel < 0.1
    params, norm, losses = closure.train(X, Y, epochs=3, lr0=3e-3, lr1=1e-3)
    assert losses[-1] < losses[0]
    err, ms, sub = closure.evaluate(setup, params, norm, steps=4, seeds=(200, 201))
    assert sub >= 1
    for k in ("uncorrected", "corrected", "uncorrected_equal_gpu_time"):
        assert len(err[k]) == 4 and all(np.isfinite(err[k])) and ms[k] > 0.0
    # the same evaluation with a fixed substep count reproduces the shared runs exactly
    err2, _, _ = closure.evaluate(setup, params, norm, steps=4, seeds=(200, 201),
                                  equal_time_substeps_n=sub)
    assert err2["uncorrected"] == err["uncorrected"] and err2["corrected"] == err["corrected"]


def test_substep_pairs_and_frontier_evaluation():
    """Coarse intervals covered by several substeps: the pair's input is the state after all of
    them (equal to stepping by hand), and evaluate_substeps applies the corrector once per
    interval (toggled on for the last substep only, which equals the substeps followed by
    dh_correct) and reports the uncorrected frontier with its GPU times."""
    setup = closure.ClosureSetup(fine=32, factor=4, runs=1, snapshots=3, spinup_steps=10, substeps=3)
    X, Y = closure.make_pairs(setup)
    assert X.shape == (3, 5, 8, 8, 8) and torch.isfinite(X).all()
    one = closure.ClosureSetup(fine=32, factor=4, runs=1, snapshots=3, spinup_steps=10, substeps=1)
    X1, Y1 = closure.make_pairs(one)
    assert torch.equal(Y, Y1)                      # same fine run and targets
    assert not torch.equal(X, X1)                  # a different coarse integration
    params = init_params(2, out_scale=1.0)
    norm = ([1.0, 0.0, 0.0, 0.0, 1.5], [0.3, 0.5, 0.5, 0.5, 0.5], [2e-3] * 5)
    # the toggled in-step correction equals three plain substeps followed by dh_correct
    shape = (16, 16, 32)
    U0 = to_gpu(inputs.decaying_turbulence(shape, seed=4, sigma=0.5, mach=0.8, p_sigma=0.2), "f32")
    a = _closure_solver(shape, params, norm)
    b = _closure_solver(shape, params, norm)
    a.init_state(U0)
    b.init_state(U0)
    for _ in range(2):
        dt = a.compute_dt()
        for j in range(3):
            a.step(dt / 3)
        a.correct()
        for j in range(3):
            b.correct_every_step(j == 2)
            b.step(dt / 3)
    assert torch.equal(a.get_state().cpu(), b.get_state().cpu())
    r = closure.evaluate_substeps(setup, params.cuda(), norm, steps=3, seeds=(200,), frontier=(1, 3))
    assert set(r["mean_error"]) == {"uncorrected_1", "uncorrected_3", "corrected"}
    assert all(np.isfinite(v) and v > 0 for v in r["mean_error"].values())
    assert r["gpu_ms_per_interval"]["uncorrected_3"] > r["gpu_ms_per_interval"]["uncorrected_1"] > 0
    assert r["equal_gpu_time_run"] in ("uncorrected_1", "uncorrected_3")


def test_non_finite_correction_is_reported_and_state_kept():
    import ctypes as C
    from paper_2512_13403_b300 import _lib
    shape = (8, 16, 16)
    U0 = inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=1.0, p_sigma=0.2)
    s = solver(shape, "f32")
    s.init_state(to_gpu(U0, "f32"))
    s.step(s.compute_dt())
    before = s.get_state().clone()
    p = torch.zeros(NPARAM, dtype=torch.float32)
    p[-5:] = 3.0e38            # output bias b3: s * y overflows to infinity
    p = p.cuda()               # kept alive across the call
    norm = (C.c_float * 15)(*([0.0] * 5 + [1.0] * 5 + [10.0] * 5))
    lib = _lib.load()
    _lib.check(lib.dh_set_corrector(s.ctx, C.c_void_p(p.data_ptr()), norm), s.ctx)
    assert lib.dh_correct(s.ctx) == 3   # DH_ERR_NONFINITE
    assert torch.equal(s.get_state(), before)
    s.step(s.compute_dt())              # the context stays usable


def test_evaluate_coarsened_self_gravitating():
    """The corrector applied at 4x coarsening of a running self-gravitating fine simulation
    (closure.evaluate_coarsened): errors against the block mean of the fine run are finite and
    positive, the fine run takes the requested steps, and a corrector whose output is zero
    leaves the corrected run on the uncorrected one (up to the floor's float32 rounding where
    cooling holds a cell at the floor energy), interval by interval."""
    from paper_2512_13403_b300.solver import Config, Solver
    n = 32
    phys = dict(forcing=True, cooling=True, t_floor=0.05, gravity=True, mg_tol=1e-6, mg_max_cycles=30)
    fine = Solver(Config(shape=(n, n, n), precision="f32", **phys))
    fine.init_state(to_gpu(inputs.self_gravitating_box((n, n, n), seed=5, sigma=0.5), "f32"))
    fine.advance(2)
    params = torch.zeros(NPARAM)
    params[:] = init_params(0, out_scale=0.0)     # output layer zero: the correction is zero
    norm = ([1.0, 0.0, 0.0, 0.0, 1.0], [0.1, 0.1, 0.1, 0.1, 0.1], [1e-3] * 5)
    ccfg = Config(shape=(n // 4,) * 3, precision="f32", **phys)
    res = closure.evaluate_coarsened(fine, ccfg, 4, params, norm, fine_steps=6)
    assert res["fine_steps"] >= 6 and res["intervals"] >= 1
    e_u, e_c = res["errors"]["uncorrected"], res["errors"]["corrected"]
    assert all(np.isfinite(e_u)) and all(e > 0 for e in e_u)
    assert np.allclose(e_c, e_u, rtol=1e-4, atol=0)
    assert res["equal_time_substeps"] >= 1
    assert all(np.isfinite(res["errors"]["uncorrected_equal_gpu_time"]))
    fine.close()


def _closure_solver(shape, params, norm, **kw):
    s = solver(shape, "f32", forcing=True, ou_seed=7, cooling=True, t_floor=0.05, **kw)
    closure._set_corrector(s, params, norm)
    return s


@pytest.mark.parametrize("gravity", [False, True])
def test_correct_every_step_matches_step_then_correct(gravity):
    """The corrector inside the step (dh_set_correct_every_step) runs the kernels of a step
    followed by dh_correct, on the device without a host synchronisation: the states, the time
    steps and the CFL step after each corrected step are bit for bit those of the explicit
    sequence."""
    shape = (16, 16, 16) if gravity else (16, 16, 32)   # gravity needs cubic cells
    U0 = to_gpu(inputs.decaying_turbulence(shape, seed=4, sigma=0.5, mach=0.8, p_sigma=0.2), "f32")
    params = init_params(2, out_scale=1.0)
    norm = ([1.0, 0.0, 0.0, 0.0, 1.5], [0.3, 0.5, 0.5, 0.5, 0.5], [2e-3] * 5)
    kw = dict(gravity=True, mg_tol=1e-6, mg_max_cycles=30) if gravity else {}
    a = _closure_solver(shape, params, norm, **kw)
    b = _closure_solver(shape, params, norm, **kw)
    a.init_state(U0)
    b.init_state(U0)
    b.correct_every_step(True)
    for _ in range(4):
        a.step(0.0)
        a.correct()
    b.advance(4)
    assert a.time() == b.time()
    assert torch.equal(a.get_state().cpu(), b.get_state().cpu())
    assert a.compute_dt() == b.compute_dt()
    # the correction did something
    c = solver(shape, "f32", forcing=True, ou_seed=7, cooling=True, t_floor=0.05, **kw)
    c.init_state(U0)
    c.advance(4)
    assert not torch.equal(c.get_state().cpu(), b.get_state().cpu())


def test_non_finite_correction_in_step_fails_the_step():
    """A corrected state that is not finite fails its step (DH_ERR_NONFINITE): the state, time
    and step count stay at the last good step, and the context keeps working once the per-step
    corrector is off.  The adjoint refuses to run while it is on."""
    from paper_2512_13403_b300 import _lib
    shape = (8, 16, 16)
    U0 = to_gpu(inputs.decaying_turbulence(shape, seed=3, sigma=0.5, mach=1.0, p_sigma=0.2), "f32")
    p = torch.zeros(NPARAM, dtype=torch.float32)
    p[-5:] = 3.0e38            # output bias b3: s * y overflows to infinity
    s = _closure_solver(shape, p, ([0.0] * 5, [1.0] * 5, [10.0] * 5))
    s.init_state(U0)
    s.advance(1)
    before, (t0, n0) = s.get_state().clone(), s.time()
    s.correct_every_step(True)
    with pytest.raises(_lib.DhError):
        s.advance(3)
    assert torch.equal(s.get_state(), before) and s.time() == (t0, n0)
    with pytest.raises(_lib.DhError):
        s.adjoint_advance(1, 1, torch.zeros_like(before))
    s.correct_every_step(False)
    s.advance(1)
    assert s.time()[1] == n0 + 1


def test_self_gravitating_pairs():
    """The self-gravitating closure set-up: solver-made pairs of runs with multigrid gravity
    from seeded lognormal densities (one per run); each pair's coarse step stays close to the
    downsampled fine run."""
    setup = closure.ClosureSetup(fine=32, factor=4, runs=2, snapshots=3, spinup_steps=3,
                                 gravity=True, sigma=0.5)
    X, Y = closure.make_pairs(setup)
    assert X.shape == (6, 5, 8, 8, 8) and torch.isfinite(X).all() and torch.isfinite(Y).all()
    assert not torch.equal(X[0], X[3])            # the two runs start from different densities
    rel = float((Y - X).norm() / Y.norm())
    assert 0.0 < rel < 0.2
