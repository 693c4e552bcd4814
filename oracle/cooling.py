"""Oracle: optically thin cooling source (Sec. 4.3) with the power-law rate Lambda = n^2 T^(1/2).

Test infrastructure only.

Readings (code units; mu m_H / k_B = 1 and R = 1):
  * n = rho, T = P / rho = (gamma - 1) E_th / rho, E_th = E - |m|^2 / (2 rho).
  * E_th floor = rho T_floor / (gamma - 1) (Sec. 4.3).  dE_th/dt = -rho^2 sqrt(T) while
    E_th > E_floor (T > T_floor), else 0; no heating.  The branch compares E_th with the floor
    energy, so a state clamped to the floor (the predictor or a substep) stops cooling exactly,
    independently of how T = (gamma-1) E_th / rho rounds.  Cells at or below the floor at the
    start of the cooling step are left untouched; elsewhere every update is max(floor, ...), so
    cooling never crosses the floor and never heats.
  * t_cool = E_th / |dE/dt| (Sec. 4.3).  N_sub = clamp(ceil(dt / (f t_cool)), 1, N_max) with
    f = 0.1, the maximum fractional change taken in the first substep, and N_max = 1024.
    N_sub = 1: trapezoid with predictor E_p = max(floor, E + dt Edot(E)),
    E_new = max(floor, E + dt/2 [Edot(E) + Edot(E_p)]).  N_sub > 1: N_sub explicit substeps
    E <- max(floor, E + Edot(E) dt/N_sub), temperature re-evaluated each substep.
  * Hitting N_max is reported as a flag; it is not an error.

Pins: tests/test_oracle_sources.py (closed form sqrt(E(t)) = sqrt(E0) - c t / 2 at fixed rho,
convergence of the subcycled update to it, floor never crossed, kinetic energy untouched,
cells below the floor unchanged).
"""
from __future__ import annotations

import math

import torch


def floor_energy(rho: torch.Tensor, gamma: float, T_floor: float) -> torch.Tensor:
    return rho * T_floor / (gamma - 1.0)


def edot(Eth: torch.Tensor, rho: torch.Tensor, gamma: float, T_floor: float) -> torch.Tensor:
    """-rho^2 sqrt(T) above the floor energy, 0 at or below it."""
    T = (gamma - 1.0) * Eth / rho
    return torch.where(Eth > floor_energy(rho, gamma, T_floor),
                       -rho * rho * torch.sqrt(torch.clamp(T, min=0.0)), torch.zeros_like(T))


def substep_count(Eth, rho, dt, gamma, T_floor, frac=0.1, nsub_max=1024):
    """Return (N_sub clamped, N_sub before the clamp) for every cell."""
    Ed = edot(Eth, rho, gamma, T_floor)
    active = Ed < 0.0
    tcool = torch.where(active, Eth / torch.where(active, -Ed, torch.ones_like(Ed)),
                        torch.full_like(Eth, math.inf))
    raw = torch.where(active, torch.ceil(dt / (frac * tcool)), torch.ones_like(Eth))
    return torch.clamp(raw, 1.0, float(nsub_max)), raw


def cool(U: torch.Tensor, dt: float, gamma: float, T_floor: float, frac: float = 0.1,
         nsub_max: int = 1024):
    """Apply one cooling step to the conserved state; returns (U_new, cap_hit)."""
    rho = U[0]
    kin = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
    Eth = U[4] - kin
    Efloor = floor_energy(rho, gamma, T_floor)
    Ed0 = edot(Eth, rho, gamma, T_floor)
    active = Ed0 < 0.0
    nsub, raw = substep_count(Eth, rho, dt, gamma, T_floor, frac, nsub_max)

    # trapezoid (N_sub = 1)
    Ep = torch.maximum(Efloor, Eth + dt * Ed0)
    Etrap = torch.maximum(Efloor, Eth + 0.5 * dt * (Ed0 + edot(Ep, rho, gamma, T_floor)))

    # subcycled (N_sub > 1), each cell with its own count
    Esub = Eth.clone()
    nmax = int(nsub.max()) if nsub.numel() else 1
    dts = dt / nsub
    for k in range(nmax):
        live = nsub > k
        Enew = torch.maximum(Efloor, Esub + edot(Esub, rho, gamma, T_floor) * dts)
        Esub = torch.where(live, Enew, Esub)

    Enew = torch.where(nsub == 1.0, Etrap, Esub)
    Enew = torch.where(active, Enew, Eth)
    out = U.clone()
    out[4] = kin + Enew
    cap_hit = bool((raw > nsub_max).any())
    return out, cap_hit


def min_cooling_time(U: torch.Tensor, gamma: float, T_floor: float) -> float:
    """min over cells of t_cool = E_th / |Edot| (Sec. 4.3), inf where nothing cools."""
    rho = U[0]
    Eth = U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
    Ed = edot(Eth, rho, gamma, T_floor)
    active = Ed < 0.0
    if not bool(active.any()):
        return math.inf
    return float((Eth[active] / (-Ed[active])).min())
