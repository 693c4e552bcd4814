"""Oracle: the hydrodynamic update of the paper (Sec. 3, Eq. 2; App. A.1-A.4).  Test infrastructure only.

State ``U``: float64 tensor of shape (5, nz, ny, nx) = (rho, m_x, m_y, m_z, E), periodic in all
three directions.  Axis ``a`` in {0, 1, 2} = {x, y, z} lives in tensor dimension ``3 - a`` of a
5-field tensor (``2 - a`` of a single field).  A face array indexed by cell ``i`` along axis a
holds the value on face i+1/2.

Readings where the paper is silent (each also listed in the design notes):
  * MC limiter: 0 if a*b <= 0 else sign(a) * min(2|a|, 2|b|, |a+b|/2), a forward and b backward
    difference (App. A.1 names the limiter only).
  * Van Leer limiter (App. A.1 lists it; the paper's fiducial runs use it): 0 if a*b <= 0 else
    2ab/(a+b), the harmonic form of the classic van Leer slope.
  * SSPRK3 (App. A.3 lists it): the Shu-Osher form U1 = U + dt L(U),
    U2 = 3/4 U + 1/4 (U1 + dt L(U1)), U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2)).
  * Positivity fallback: if either reconstructed face state of a cell along an axis has
    rho <= 0 or P <= 0, all slopes of that cell along that axis are set to zero.
  * HLLC: Toro-Spruce-Speares star states with the Davis wave speeds of App. A.2; region
    choice SL >= 0 -> F_L, else S* >= 0 -> F*_L, else SR > 0 -> F*_R, else F_R.
  * CFL (App. A.4): dt = C * min over cells and axes of dx_a / (|v_a| + c_s).

Pins: tests/test_oracle_hydro.py (hand HLLC values, MC truth table, EOS round trip, exact Sod
solution, second-order sound-wave convergence, conservation, axis symmetry, dt hand value).
"""
from __future__ import annotations

import torch

NFIELD = 5


def _dim(axis: int, nfield_leading: bool = True) -> int:
    return 3 - axis if nfield_leading else 2 - axis


def cons_to_prim(U: torch.Tensor, gamma: float) -> torch.Tensor:
    """W = (rho, v, P) from U = (rho, rho v, E): v = m / rho, P = (gamma-1)(E - rho |v|^2 / 2) (Eq. 2)."""
    rho = U[0]
    vx = U[1] / rho
    vy = U[2] / rho
    vz = U[3] / rho
    P = (gamma - 1.0) * (U[4] - 0.5 * rho * (vx * vx + vy * vy + vz * vz))
    return torch.stack([rho, vx, vy, vz, P])


def prim_to_cons(W: torch.Tensor, gamma: float) -> torch.Tensor:
    """Inverse of cons_to_prim (Eq. 2)."""
    rho, vx, vy, vz, P = W
    E = P / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return torch.stack([rho, rho * vx, rho * vy, rho * vz, E])


def mc_limiter(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Monotonized-central slope from forward difference a and backward difference b (App. A.1)."""
    mag = torch.minimum(torch.minimum(2.0 * a.abs(), 2.0 * b.abs()), 0.5 * (a + b).abs())
    slope = torch.sign(a) * mag
    return torch.where(a * b > 0.0, slope, torch.zeros_like(slope))


def van_leer_limiter(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Van Leer slope 2ab/(a+b) where a*b > 0, else 0 (App. A.1).  The denominator of the branch
    not taken is replaced by 1 so that reverse mode sees no 0/0 there."""
    pos = a * b > 0.0
    den = torch.where(pos, a + b, torch.ones_like(a))
    return torch.where(pos, 2.0 * a * b / den, torch.zeros_like(a))


LIMITERS = {"mc": mc_limiter, "vanleer": van_leer_limiter}


def limited_slopes(W: torch.Tensor, axis: int, limiter: str = "mc") -> torch.Tensor:
    """Delta W_i = lim(W_{i+1} - W_i, W_i - W_{i-1}) per primitive, with the positivity fallback."""
    d = _dim(axis)
    Wp = torch.roll(W, -1, dims=d)
    Wm = torch.roll(W, 1, dims=d)
    dW = LIMITERS[limiter](Wp - W, W - Wm)
    hi = W + 0.5 * dW
    lo = W - 0.5 * dW
    bad = (hi[0] <= 0.0) | (hi[4] <= 0.0) | (lo[0] <= 0.0) | (lo[4] <= 0.0)
    return torch.where(bad.unsqueeze(0), torch.zeros_like(dW), dW)


def face_states(W: torch.Tensor, axis: int, limiter: str = "mc"):
    """W^L_{i+1/2} = W_i + dW_i / 2 and W^R_{i+1/2} = W_{i+1} - dW_{i+1} / 2 (App. A.1)."""
    dW = limited_slopes(W, axis, limiter)
    WL = W + 0.5 * dW
    WR = torch.roll(W - 0.5 * dW, -1, dims=_dim(axis))
    return WL, WR


def _normal_tangential(axis: int):
    """Velocity slots (1..3) as (normal, tangential_1, tangential_2) for a face normal to axis."""
    n = 1 + axis
    t = [1 + a for a in range(3) if a != axis]
    return n, t[0], t[1]


def physical_flux(W: torch.Tensor, axis: int, gamma: float) -> torch.Tensor:
    """Euler flux along axis: (rho u, rho u v + P e_n, u (E + P)) with u the normal velocity."""
    rho, P = W[0], W[4]
    n = 1 + axis
    u = W[n]
    E = P / (gamma - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3])
    F = [rho * u, rho * u * W[1], rho * u * W[2], rho * u * W[3], u * (E + P)]
    F[n] = F[n] + P
    return torch.stack(F)


def _safe_div(a, b):
    return a / torch.where(b == 0.0, torch.ones_like(b), b)


def hllc_flux(WL: torch.Tensor, WR: torch.Tensor, axis: int, gamma: float) -> torch.Tensor:
    """HLLC flux across faces normal to ``axis`` (App. A.2; Toro, Spruce & Speares 1994).

    Wave speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R), c^2 = gamma P / rho.
    """
    n, t1, t2 = _normal_tangential(axis)
    rL, uL, PL = WL[0], WL[n], WL[4]
    rR, uR, PR = WR[0], WR[n], WR[4]
    cL = torch.sqrt(gamma * PL / rL)
    cR = torch.sqrt(gamma * PR / rR)
    SL = torch.minimum(uL - cL, uR - cR)
    SR = torch.maximum(uL + cL, uR + cR)

    UL = prim_to_cons(WL, gamma)
    UR = prim_to_cons(WR, gamma)
    FL = physical_flux(WL, axis, gamma)
    FR = physical_flux(WR, axis, gamma)

    Sstar = (PR - PL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (
        rL * (SL - uL) - rR * (SR - uR))

    def star_flux(WK, UK, FK, SK):
        rK, uK, PK = WK[0], WK[n], WK[4]
        coef = _safe_div(rK * (SK - uK), SK - Sstar)
        Us = [None] * 5
        Us[0] = coef
        Us[n] = coef * Sstar
        Us[t1] = coef * WK[t1]
        Us[t2] = coef * WK[t2]
        Us[4] = coef * (UK[4] / rK + (Sstar - uK) * (Sstar + _safe_div(PK, rK * (SK - uK))))
        return FK + SK * (torch.stack(Us) - UK)

    FsL = star_flux(WL, UL, FL, SL)
    FsR = star_flux(WR, UR, FR, SR)
    return torch.where(SL >= 0.0, FL,
                       torch.where(Sstar >= 0.0, FsL,
                                   torch.where(SR > 0.0, FsR, FR)))


def rhs(U: torch.Tensor, gamma: float, dx, limiter: str = "mc") -> torch.Tensor:
    """Unsplit method-of-lines RHS dU/dt = -sum_a (F_a,i+1/2 - F_a,i-1/2) / dx_a (App. A.3)."""
    W = cons_to_prim(U, gamma)
    L = torch.zeros_like(U)
    for axis in range(3):
        WL, WR = face_states(W, axis, limiter)
        F = hllc_flux(WL, WR, axis, gamma)
        L = L - (F - torch.roll(F, 1, dims=_dim(axis))) / dx[axis]
    return L


def rk2_step(U: torch.Tensor, dt: float, gamma: float, dx, limiter: str = "mc") -> torch.Tensor:
    """Heun / SSP-RK2 (App. A.3): U1 = U + dt L(U); U^{n+1} = U/2 + (U1 + dt L(U1))/2."""
    U1 = U + dt * rhs(U, gamma, dx, limiter)
    return 0.5 * U + 0.5 * (U1 + dt * rhs(U1, gamma, dx, limiter))


def ssprk3(L, U: torch.Tensor, dt: float) -> torch.Tensor:
    """Shu-Osher SSPRK3 for dU/dt = L(U) (App. A.3)."""
    U1 = U + dt * L(U)
    U2 = 0.75 * U + 0.25 * (U1 + dt * L(U1))
    return U / 3.0 + (2.0 / 3.0) * (U2 + dt * L(U2))


def ssprk3_step(U: torch.Tensor, dt: float, gamma: float, dx, limiter: str = "mc") -> torch.Tensor:
    return ssprk3(lambda V: rhs(V, gamma, dx, limiter), U, dt)


def step(U: torch.Tensor, dt: float, gamma: float, dx, integrator: str = "rk2",
         limiter: str = "mc") -> torch.Tensor:
    """The hydro update of one step with the chosen integrator and limiter."""
    if integrator == "rk2":
        return rk2_step(U, dt, gamma, dx, limiter)
    if integrator == "ssprk3":
        return ssprk3_step(U, dt, gamma, dx, limiter)
    raise ValueError(integrator)


def rk2_stages(U: torch.Tensor, dt: float, gamma: float, dx):
    """Both RK2 stage results (U1, U^{n+1}) for stage-by-stage comparisons."""
    U1 = U + dt * rhs(U, gamma, dx)
    return U1, 0.5 * U + 0.5 * (U1 + dt * rhs(U1, gamma, dx))


def euler_step(U: torch.Tensor, dt: float, gamma: float, dx) -> torch.Tensor:
    """First-order forward Euler in time (App. A.3, the testing integrator)."""
    return U + dt * rhs(U, gamma, dx)


def cfl_dt(U: torch.Tensor, gamma: float, dx, cfl: float) -> float:
    """dt = C * min over cells and axes of dx_a / (|v_a| + c_s) (App. A.4)."""
    W = cons_to_prim(U, gamma)
    cs = torch.sqrt(gamma * W[4] / W[0])
    m = None
    for axis in range(3):
        t = dx[axis] / (W[1 + axis].abs() + cs)
        tm = t.min()
        m = tm if m is None else torch.minimum(m, tm)
    return float(cfl * m)


def conserved_totals(U: torch.Tensor):
    """Sum over cells of each conserved field, exactly rounded (math.fsum) in float64."""
    import math
    return [math.fsum(U[f].reshape(-1).tolist()) for f in range(NFIELD)]
