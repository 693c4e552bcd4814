"""Oracle: vector-Jacobian products of the hydro step with the time step held fixed.

Test infrastructure only.  The product J^T lambda of the discrete RK2 step (App. A.3) is
obtained by reverse-mode differentiation of the oracle's own forward step (``hydro.rk2_step``),
which is its definition; dt is a constant (the "stopped" time-step gradient of App. A.4).  At a
kink the derivative is that of the branch the forward took (torch's one-sided rules; the
limiter's a*b <= 0 branch has zero derivative).  Long integrations recompute each step from the
stored states (checkpointing in its simplest form, Sec. 2.3).

Pins: tests/test_oracle_adjoint.py (central finite differences, the dot-product identity with
forward-mode products, and the exact mass invariant dL/drho_0 = 1/N^3 for L = mean(rho_final)).
"""
from __future__ import annotations

import torch

from . import hydro as _hydro


def step_vjp(U: torch.Tensor, dt: float, lam: torch.Tensor, gamma: float, dx, a=None):
    """lambda^n = (dU^{n+1}/dU^n)^T lambda^{n+1} for one RK2 step (+ optional fixed forcing a)."""
    Ud = U.detach().clone().requires_grad_(True)
    out = _hydro.rk2_step(Ud, dt, gamma, dx)
    if a is not None:
        kick = out.clone()
        kick[1:4] = out[1:4] + out[0] * a * dt
        kick[4] = out[4] + (out[1] * a[0] + out[2] * a[1] + out[3] * a[2]) * dt
        out = kick
    (g,) = torch.autograd.grad(out, Ud, grad_outputs=lam)
    return g


def advance_vjp(U0: torch.Tensor, dts, lam_final: torch.Tensor, gamma: float, dx):
    """lambda^0 for U^n = H_{dt_{n-1}} o ... o H_{dt_0}(U^0); states recomputed forward first."""
    states = [U0.detach().clone()]
    with torch.no_grad():
        for dt in dts[:-1]:
            states.append(_hydro.rk2_step(states[-1], dt, gamma, dx))
    lam = lam_final.clone()
    for n in reversed(range(len(dts))):
        lam = step_vjp(states[n], dts[n], lam, gamma, dx)
    return lam


def advance(U0: torch.Tensor, dts, gamma: float, dx) -> torch.Tensor:
    U = U0.clone()
    for dt in dts:
        U = _hydro.rk2_step(U, dt, gamma, dx)
    return U
