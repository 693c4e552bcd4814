"""GPU flux-form corrector, the network's vector-Jacobian product and the solver-in-the-loop
rollout gradient (Sec. 7) against reverse mode of the oracle.

The oracle's BF16 roundings are passed straight through in reverse mode (the GPU treats them as
the identity in its VJP), so forward values carry the BF16 rounding and gradients do not; the
comparisons use the tolerances of the network's other GPU tests (1e-2 on values, 3e-2 on
gradients)."""
import numpy as np
import pytest
import torch

from oracle import corrector as oc
from oracle import hydro as ohydro
from paper_2512_13403_b300 import inputs
from tests.gpu_util import solver, to_gpu

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _straight_through(monkeypatch):
    monkeypatch.setattr(oc, "bf16", lambda t: t + (t.to(torch.bfloat16).to(torch.float64) - t).detach())


def _params(form, seed):
    from paper_2512_13403_b300 import corrector as cr
    p = cr.init_params(seed, out_scale=1.0, form=form)
    p = p + 0.01 * torch.randn(p.shape, generator=torch.Generator().manual_seed(seed))
    return p, cr.unflatten(p.double())


def _compared(form):
    """Parameter blocks compared by relative error.  In the flux form the output bias is a
    constant flux, which has no divergence: its gradient is exactly zero and checked apart."""
    return ("W1", "b1", "W2", "b2", "W3") + (("b3",) if form == "state" else ())


def _state(shape, seed=1):
    return torch.from_numpy(inputs.decaying_turbulence(shape, seed=seed, sigma=0.5, mach=1.0, p_sigma=0.3))


def _rel(a, b):
    a = torch.as_tensor(a).double().cpu()
    b = torch.as_tensor(b).double().cpu()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("form", ["state", "flux"])
def test_correction_matches_oracle_and_flux_form_conserves(form, monkeypatch):
    from paper_2512_13403_b300 import corrector as cr
    _straight_through(monkeypatch)
    shape = (8, 12, 16)
    params, pd = _params(form, 3)
    U = _state(shape)
    mu = [float(U[c].mean()) for c in range(5)]
    sigma = [float(U[c].std()) for c in range(5)]
    out = [0.01 * s for s in sigma]
    net = cr.Network(shape, form=form)
    net.set_params(params, mu, sigma, out)
    Ug = U.float().cuda().contiguous()
    V = Ug.clone()
    net.correct_state(V, 1e-9, 1e-6, G)
    ref = oc.correct(Ug.double().cpu(), pd, mu, sigma, 1e-9, 1e-6, G, out)
    assert _rel(V - Ug, ref - Ug.double().cpu()) < 1e-2
    tot0 = Ug.double().sum(dim=(1, 2, 3)).cpu()
    tot1 = V.double().sum(dim=(1, 2, 3)).cpu()
    if form == "flux":
        # a divergence moves the totals only by float32 rounding of the update
        scale = Ug.double().abs().sum(dim=(1, 2, 3)).cpu()
        assert torch.all((tot1 - tot0).abs() <= 1e-6 * scale), (tot1 - tot0) / scale
    else:
        assert float((tot1 - tot0).abs().max()) > 0.0
    net.close()


@pytest.mark.parametrize("form", ["state", "flux"])
def test_vjp_matches_oracle(form, monkeypatch):
    """dh_cnn_vjp: parameter and input gradients of <g, dU(U)> for an upstream gradient g."""
    from paper_2512_13403_b300 import corrector as cr
    _straight_through(monkeypatch)
    shape = (8, 12, 16)
    params, pd = _params(form, 5)
    U = _state(shape, seed=2)
    mu = [float(U[c].mean()) for c in range(5)]
    sigma = [float(U[c].std()) for c in range(5)]
    out = [0.5 * s for s in sigma]
    net = cr.Network(shape, form=form)
    net.set_params(params, mu, sigma, out)
    Ug = U.float().cuda().contiguous()
    g = torch.randn((5,) + shape, generator=torch.Generator().manual_seed(11), dtype=torch.float64)
    net.forward(Ug)
    grads = torch.zeros(cr.nparam(form), dtype=torch.float32, device="cuda")
    gU = net.vjp(g.float().cuda().contiguous(), grads)
    q = {k: v.clone().requires_grad_(True) for k, v in pd.items()}
    Uq = Ug.double().cpu().requires_grad_(True)
    (oc.correction(Uq, q, mu, sigma, out) * g).sum().backward()
    gg = cr.unflatten(grads.double().cpu())
    for k in _compared(form):
        assert _rel(gg[k], q[k].grad) < 3e-2, k
    if form == "flux":
        assert float(gg["b3"].abs().max()) == 0.0 and float(q["b3"].grad.abs().max()) < 1e-12
    assert _rel(gU, Uq.grad) < 3e-2
    net.close()


def test_flux_form_one_step_backward_matches_oracle(monkeypatch):
    """dh_cnn_backward in the flux form: mean squared error of the divergence against the
    residual target."""
    from paper_2512_13403_b300 import corrector as cr
    _straight_through(monkeypatch)
    shape = (8, 12, 16)
    params, pd = _params("flux", 7)
    U = _state(shape, seed=4)
    mu = [float(U[c].mean()) for c in range(5)]
    sigma = [float(U[c].std()) for c in range(5)]
    out = [0.2 * s for s in sigma]
    net = cr.Network(shape, form="flux")
    net.set_params(params, mu, sigma, out)
    Ug = U.float().cuda().contiguous()
    T = (Ug + 0.05 * torch.randn(Ug.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3))).contiguous()
    net.forward(Ug)
    grads = torch.zeros(cr.nparam("flux"), dtype=torch.float32, device="cuda")
    loss = net.backward(Ug, T, grads)
    q = {k: v.clone().requires_grad_(True) for k, v in pd.items()}
    s = torch.tensor(out, dtype=torch.float64).reshape(5, 1, 1, 1)
    t = (T.double().cpu() - Ug.double().cpu()) / s
    y, _ = oc.forward(Ug.double().cpu(), q, mu, sigma)
    L = ((oc.flux_divergence(y) - t) ** 2).mean()
    L.backward()
    assert loss == pytest.approx(float(L.detach()), rel=2e-2)
    gg = cr.unflatten(grads.double().cpu())
    for k in _compared("flux"):
        assert _rel(gg[k], q[k].grad) < 3e-2, k
    assert float(gg["b3"].abs().max()) == 0.0
    net.close()


@pytest.mark.parametrize("form,floors,substeps", [("state", False, 1), ("flux", False, 1),
                                                  ("state", True, 1), ("flux", True, 1),
                                                  ("state", False, 2)])
def test_rollout_gradient_matches_oracle(form, floors, substeps, monkeypatch):
    """The rollout loss and its parameter gradient through two intervals of one or two solver
    steps each (hand adjoint, imposed dt) and two corrections, against reverse mode of the oracle
    rollout.  With
    `floors`, rho_floor = 0.9 <rho> and T_floor = 0.6 bind in a large share of the cells (both
    the density floor and the energy floor), and the gradient goes through them."""
    from paper_2512_13403_b300 import closure
    from paper_2512_13403_b300.solver import Config
    _straight_through(monkeypatch)
    shape = (16, 16, 16)
    U0 = inputs.decaying_turbulence(shape, seed=6, sigma=0.3, mach=0.6, p_sigma=0.2)
    U0t = torch.from_numpy(U0)
    dx = (1 / 16, 1 / 16, 1 / 16)
    dts = [0.9 * ohydro.cfl_dt(U0t, G, dx, 0.4)] * 2
    targets = [U0t + 0.02 * torch.randn(U0t.shape, generator=torch.Generator().manual_seed(k), dtype=torch.float64)
               for k in (1, 2)]
    params, pd = _params(form, 9)
    mu = [float(U0t[c].mean()) for c in range(5)]
    sigma = [float(U0t[c].std()) for c in range(5)]
    out = [0.02 * s for s in sigma]
    w = [float(U0t[c].std()) for c in range(5)]
    frac = 0.9 if floors else 1e-9
    cfg = Config(shape=shape, precision="f32", t_floor=0.6 if floors else 0.05)
    tr = closure.RolloutTrainer(shape, cfg, form, rho_floor_frac=frac, substeps=substeps)
    traj = closure.Trajectory(to_gpu(U0, "f32"), dts, [None, None],
                              [t.float().cuda().contiguous() for t in targets])
    L, g = tr.loss_and_grad(traj, params.cuda(), (mu, sigma, out), w)
    tr.close()
    q = {k: v.clone().requires_grad_(True) for k, v in pd.items()}
    def interval(U, dt):   # `substeps` equal solver steps per interval
        for _ in range(substeps):
            U = ohydro.rk2_step(U, dt / substeps, G, dx)
        return U
    steps = [lambda U, dt=dt: interval(U, dt) for dt in dts]
    rho_floor = frac * float(U0t[0].mean())
    Lr = oc.rollout_loss(U0t, steps, targets, q, mu, sigma, out, w, rho_floor, cfg.t_floor, G)
    Lr.backward()
    if floors:
        # the floors do bind: the corrected state differs from the unfloored one in many cells
        with torch.no_grad():
            V = steps[0](U0t)
            Y = V + oc.correction(V, pd, mu, sigma, out)
            Z = oc.correct(V, pd, mu, sigma, rho_floor, cfg.t_floor, G, out)
            assert int((Z[0] != Y[0]).sum()) > 100 and int((Z[4] != Y[4]).sum()) > 100
    assert L == pytest.approx(float(Lr.detach()), rel=1e-2)
    from paper_2512_13403_b300 import corrector as cr
    gg = cr.unflatten(g.double().cpu())
    for k in _compared(form):
        assert _rel(gg[k], q[k].grad) < 3e-2, k


def test_adjoint_with_imposed_dt_matches_oracle():
    shape = (12, 10, 20)
    U0 = inputs.decaying_turbulence(shape, seed=5, sigma=0.3, mach=0.8, p_sigma=0.3)
    lam = np.random.default_rng(1).standard_normal((5,) + shape)
    dx = (1 / 20, 1 / 10, 1 / 12)
    dt = 0.7 * ohydro.cfl_dt(torch.from_numpy(U0), G, dx, 0.4)
    s = solver(shape, "f64")
    s.init_state(to_gpu(U0, "f64"))
    gpu = s.adjoint_advance(3, 2, to_gpu(lam, "f64"), dt=dt)
    from oracle import adjoint as oadj
    ref = oadj.advance_vjp(torch.from_numpy(U0), [dt] * 3, torch.from_numpy(lam), G, dx)
    assert _rel(gpu, ref) < 1e-10
    assert s.time()[0] == pytest.approx(3 * dt, rel=1e-14)
