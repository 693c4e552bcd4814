"""Oracle: one full step of the method (Sec. 2.1 update H; App. A.3-A.4; Secs. 3.1.1, 4.3, 5.2).

Test infrastructure only.

Order of one step from state U^n (readings where the paper does not fix the order):
  1. dt: the caller's value, else C * min dx_a / (|v_a| + c_s) (App. A.4), further limited by
     c_cool * min t_cool and dt_max when those are finite (Sec. 4.3).
  2. OU forcing (if on): advance the mode table by dt (Sec. 3.1.1) and synthesise a(x).
  3. Hydro: SSP-RK2 over the unsplit RHS (App. A.3).
  4. Sources, Lie-split after the hydro update in the order forcing -> gravity -> cooling, each on
     the state left by the previous one; gravity solves the Poisson problem on rho after step 3.
  5. t += dt.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import torch

from . import cooling as _cool
from . import forcing as _force
from . import hydro as _hydro
from . import multigrid as _mg


@dataclasses.dataclass
class Config:
    shape: Tuple[int, int, int]                 # (nz, ny, nx)
    dx: Tuple[float, float, float] = None       # (dx, dy, dz); default 1/N per axis (unit box)
    gamma: float = 5.0 / 3.0
    cfl: float = 0.4
    forcing: bool = False
    ou_tau: float = 0.5
    ou_arms: float = 1.0
    ou_seed: int = 1
    cooling: bool = False
    t_floor: float = 0.05
    cool_frac: float = 0.1
    nsub_max: int = 1024
    c_cool: float = math.inf
    dt_max: float = math.inf
    gravity: bool = False
    four_pi_G: float = 1.0
    mg_tol: float = 1e-6
    mg_max_cycles: int = 30
    mg_pre: int = 2
    mg_post: int = 2
    integrator: str = "rk2"       # "rk2" or "ssprk3"
    limiter: str = "mc"           # "mc" or "vanleer"
    mg_smoother: str = "rbgs"
    mg_omega: float = 2.0 / 3.0
    mg_cycle: str = "V"

    def __post_init__(self):
        if self.dx is None:
            nz, ny, nx = self.shape
            self.dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)


class Simulation:
    def __init__(self, cfg: Config, U0):
        self.cfg = cfg
        self.U = torch.as_tensor(U0, dtype=torch.float64).clone()
        assert tuple(self.U.shape[1:]) == tuple(cfg.shape)
        self.t = 0.0
        self.nstep = 0
        self.ou = _force.OUForcing(cfg.ou_seed, cfg.ou_tau, cfg.ou_arms) if cfg.forcing else None
        self.phi = torch.zeros(cfg.shape, dtype=torch.float64) if cfg.gravity else None
        self.mg_cycles = 0
        self.mg_residual = 0.0
        self.cool_cap_hit = False

    def compute_dt(self) -> float:
        c = self.cfg
        dt = _hydro.cfl_dt(self.U, c.gamma, c.dx, c.cfl)
        if c.cooling and math.isfinite(c.c_cool):
            dt = min(dt, c.c_cool * _cool.min_cooling_time(self.U, c.gamma, c.t_floor))
        return min(dt, c.dt_max)

    def step(self, dt: Optional[float] = None) -> float:
        c = self.cfg
        if dt is None or dt <= 0.0:
            dt = self.compute_dt()
        a = None
        if self.ou is not None:
            self.ou.update(dt, self.nstep)
            a = self.ou.field(c.shape)
        self.last_field = a
        U = _hydro.step(self.U, dt, c.gamma, c.dx, c.integrator, c.limiter)
        if a is not None:
            U = _force.apply_forcing(U, a, dt)
        if c.gravity:
            F = _mg.poisson_source(U[0], c.four_pi_G)
            self.phi, self.mg_cycles, self.mg_residual, ok = _mg.solve(
                F, c.dx[0], self.phi, c.mg_tol, c.mg_max_cycles, c.mg_pre, c.mg_post,
                c.mg_smoother, c.mg_omega, c.mg_cycle)
            U = _mg.gravity_source(U, self.phi, dt, c.dx[0])
        if c.cooling:
            U, cap = _cool.cool(U, dt, c.gamma, c.t_floor, c.cool_frac, c.nsub_max)
            self.cool_cap_hit = self.cool_cap_hit or cap
        self.U = U
        self.t += dt
        self.nstep += 1
        return dt

    def advance(self, nsteps: int):
        dts = []
        for _ in range(nsteps):
            dts.append(self.step())
        return dts
