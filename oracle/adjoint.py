"""Oracle: vector-Jacobian products of the hydro step with the time step held fixed.

Test infrastructure only.  The product J^T lambda of the discrete RK2 step (App. A.3) is
obtained by reverse-mode differentiation of the oracle's own forward step (``hydro.rk2_step``),
which is its definition; dt is a constant (the "stopped" time-step gradient of App. A.4).  At a
kink the derivative is that of the branch the forward took (torch's one-sided rules; the
limiter's a*b <= 0 branch has zero derivative).  Long integrations recompute each step from the
stored states (checkpointing in its simplest form, Sec. 2.3).

With sources the step is RK2, then the forcing kick with the step's field held fixed (it depends
on the random draws only), then self-gravity with the exact Poisson solution of the seven-point
operator (the limit of the V-cycles; differentiated through the FFT solve), then cooling,
differentiated through the oracle's own cooling routine (the branch the forward took; the
integer substep count carries no derivative).

Pins: tests/test_oracle_adjoint.py (central finite differences, the dot-product identity with
forward-mode products, and the exact mass invariant dL/drho_0 = 1/N^3 for L = mean(rho_final),
with and without forcing and cooling).
"""
from __future__ import annotations

import torch

from . import cooling as _cool
from . import forcing as _force
from . import hydro as _hydro
from . import multigrid as _mg


def full_step(U: torch.Tensor, dt: float, gamma: float, dx, a=None, cooling=None,
              gravity=None, scheme=None) -> torch.Tensor:
    """One step as the driver takes it: RK2 (App. A.3), then the Lie-split sources in their
    order, the forcing kick with the fixed field a (Sec. 3.1.1), self-gravity (Sec. 5:
    `gravity` = dict(four_pi_G=) or None, phi the exact solution of the seven-point Poisson
    problem, which converged V-cycles reproduce to their tolerance) and cooling (Sec. 4.3;
    `cooling` = dict(T_floor=, frac=, nsub_max=) or None).  `scheme` = dict(integrator=,
    limiter=) or None (RK2 with MC)."""
    U = _hydro.step(U, dt, gamma, dx, **(scheme or {}))
    if a is not None:
        U = _force.apply_forcing(U, a, dt)
    if gravity is not None:
        phi = _mg.fft_solve(_mg.poisson_source(U[0], gravity["four_pi_G"]), dx[0])
        U = _mg.gravity_source(U, phi, dt, dx[0])
    if cooling is not None:
        U, _ = _cool.cool(U, dt, gamma, cooling["T_floor"], cooling.get("frac", 0.1),
                          cooling.get("nsub_max", 1024))
    return U


def step_vjp(U: torch.Tensor, dt: float, lam: torch.Tensor, gamma: float, dx, a=None,
             cooling=None, gravity=None, scheme=None):
    """lambda^n = (dU^{n+1}/dU^n)^T lambda^{n+1} for one step (sources optional)."""
    Ud = U.detach().clone().requires_grad_(True)
    out = full_step(Ud, dt, gamma, dx, a, cooling, gravity, scheme)
    (g,) = torch.autograd.grad(out, Ud, grad_outputs=lam)
    return g


def advance_vjp(U0: torch.Tensor, dts, lam_final: torch.Tensor, gamma: float, dx, fields=None,
                cooling=None, gravity=None, scheme=None):
    """lambda^0 for U^n = H_{n-1} o ... o H_0(U^0) (fields[n]: forcing of step n, or None);
    states recomputed forward first."""
    fields = fields if fields is not None else [None] * len(dts)
    states = [U0.detach().clone()]
    with torch.no_grad():
        for n in range(len(dts) - 1):
            states.append(full_step(states[-1], dts[n], gamma, dx, fields[n], cooling, gravity,
                                    scheme))
    lam = lam_final.clone()
    for n in reversed(range(len(dts))):
        lam = step_vjp(states[n], dts[n], lam, gamma, dx, fields[n], cooling, gravity, scheme)
    return lam


def advance(U0: torch.Tensor, dts, gamma: float, dx, fields=None, cooling=None,
            gravity=None, scheme=None) -> torch.Tensor:
    fields = fields if fields is not None else [None] * len(dts)
    U = U0.clone()
    for n, dt in enumerate(dts):
        U = full_step(U, dt, gamma, dx, fields[n], cooling, gravity, scheme)
    return U


def record(sim, nsteps: int):
    """Runs an oracle Simulation for nsteps CFL steps; returns (dts, forcing fields per step)."""
    dts, fields = [], []
    for _ in range(nsteps):
        dts.append(sim.step())
        fields.append(sim.last_field)
    return dts, fields
