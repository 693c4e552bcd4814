"""Oracle: Ornstein-Uhlenbeck turbulent forcing (Sec. 3.1.1).  Test infrastructure only.

Readings of what the section leaves open:
  * Forced modes: integer n with 1 <= |n|^2 <= 4 (the band 1 <= |k| L / 2 pi <= 2).  The field
    is stored on the half-space H = {first nonzero component of n > 0} (16 modes, ordered
    lexicographically by (n_x, n_y, n_z)); the other half follows from a(x) being real.
  * Flat amplitude across the band, purely solenoidal projection P_ij = delta_ij - n_i n_j / |n|^2
    (zeta = 1), applied to the Gaussian draw; the k = 0 mode is never present.
  * Gaussian draws: a counter-based SplitMix64 stream.  key = splitmix64(seed); the i-th
    64-bit word is splitmix64(key + i * 0x9E3779B97F4A7C15) (mod 2^64), i.e. output i of the
    SplitMix64 generator started at state ``key``; u = ((word >> 11) + 0.5) * 2^-53.  Draw d,
    mode m, component c uses words i = 2 * ((d * 16 + m) * 3 + c) and i + 1 for a Box-Muller
    pair: real part sqrt(-2 ln u1) cos(2 pi u2), imaginary part sqrt(-2 ln u1) sin(2 pi u2).
  * Draw d = 0 initialises the state (stationary start: a_hat = P xi_0); the update taken
    during step s (s = 0, 1, ...) uses draw d = s + 1.
  * Synthesis: a(x) = 2 Re sum_{n in H} a_hat_n exp(2 pi i n . x~), x~_a = (i_a + 1/2) / N_a.
  * Normalisation: a -> a * a_rms / sqrt(<|a|^2>) with <|a|^2> = 2 sum_H |a_hat|^2 (Parseval on
    the grid, exact when every N_a >= 5 so the forced modes do not alias).
  * Coupling: dm = rho a dt, dE = (m . a) dt with m taken before the kick.

Pins: tests/test_oracle_sources.py (Parseval against a brute-force mean, zero divergence
n . a_hat = 0, zero mean, stationary variance of the recurrence, the SplitMix64 reference
outputs of its published test vector, Box-Muller moments, exact momentum kick with u = 0).
"""
from __future__ import annotations

import math

import torch

MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15
NMODE = 16


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014): one increment then the mixer."""
    z = (x + GOLDEN64) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream_word(key: int, i: int) -> int:
    return splitmix64((key + i * GOLDEN64) & MASK64)


def unit_uniform(word: int) -> float:
    return ((word >> 11) + 0.5) * (2.0 ** -53)


def forced_modes():
    """Half-space integer modes with 1 <= |n|^2 <= 4, lexicographic in (n_x, n_y, n_z)."""
    modes = []
    for nx in range(-2, 3):
        for ny in range(-2, 3):
            for nz in range(-2, 3):
                k2 = nx * nx + ny * ny + nz * nz
                if not (1 <= k2 <= 4):
                    continue
                first = nx if nx != 0 else (ny if ny != 0 else nz)
                if first > 0:
                    modes.append((nx, ny, nz))
    assert len(modes) == NMODE
    return modes


def gaussian_draw(seed: int, draw: int) -> torch.Tensor:
    """Complex standard normals xi[m, c] (real+imag each N(0,1)) for one draw index."""
    key = splitmix64(seed & MASK64)
    xi = torch.zeros(NMODE, 3, dtype=torch.complex128)
    for m in range(NMODE):
        for c in range(3):
            i0 = 2 * ((draw * NMODE + m) * 3 + c)
            u1 = unit_uniform(stream_word(key, i0))
            u2 = unit_uniform(stream_word(key, i0 + 1))
            r = math.sqrt(-2.0 * math.log(u1))
            th = 2.0 * math.pi * u2
            xi[m, c] = complex(r * math.cos(th), r * math.sin(th))
    return xi


def solenoidal_projection(xi: torch.Tensor) -> torch.Tensor:
    """eta_i = (delta_ij - n_i n_j / |n|^2) xi_j per mode (Sec. 3.1, tensor P)."""
    n = torch.tensor(forced_modes(), dtype=torch.float64)
    k2 = (n * n).sum(1, keepdim=True)
    proj = torch.eye(3, dtype=torch.float64)[None] - n[:, :, None] * n[:, None, :] / k2[:, :, None]
    return torch.einsum('mij,mj->mi', proj.to(torch.complex128), xi)


class OUForcing:
    """Mode table a_hat[m, c] of the OU process and its real-space field."""

    def __init__(self, seed: int, tau: float, a_rms: float):
        self.seed = seed
        self.tau = tau
        self.a_rms = a_rms
        self.a_hat = solenoidal_projection(gaussian_draw(seed, 0))

    def update(self, dt: float, step_index: int):
        """a_hat <- exp(-dt/tau) a_hat + sqrt(1 - exp(-2 dt/tau)) eta (Sec. 3.1.1)."""
        f = math.exp(-dt / self.tau)
        eta = solenoidal_projection(gaussian_draw(self.seed, step_index + 1))
        self.a_hat = f * self.a_hat + math.sqrt(1.0 - f * f) * eta

    def mean_square(self) -> float:
        """<|a|^2> over the grid by Parseval: 2 sum over H and components of |a_hat|^2."""
        return float(2.0 * (self.a_hat.abs() ** 2).sum())

    def raw_field(self, shape) -> torch.Tensor:
        """Unnormalised a(x) on the cell centres, shape (3, nz, ny, nx)."""
        nz, ny, nx = shape
        xs = [(torch.arange(n, dtype=torch.float64) + 0.5) / n for n in (nx, ny, nz)]
        a = torch.zeros((3, nz, ny, nx), dtype=torch.float64)
        for m, (mx, my, mz) in enumerate(forced_modes()):
            phase = 2.0 * math.pi * (mx * xs[0][None, None, :] + my * xs[1][None, :, None]
                                     + mz * xs[2][:, None, None])
            e = torch.exp(1j * phase)
            for c in range(3):
                a[c] += 2.0 * (self.a_hat[m, c] * e).real
        return a

    def field(self, shape) -> torch.Tensor:
        """a(x) normalised to the prescribed rms amplitude (Sec. 3.1.1)."""
        return self.raw_field(shape) * (self.a_rms / math.sqrt(self.mean_square()))

    def field_at(self, shape, k: torch.Tensor, j: torch.Tensor, i: torch.Tensor) -> torch.Tensor:
        """The normalised a(x) of `field` at the cells (k, j, i) only (integer tensors of one
        shape), shape (3,) + k.shape: the same sum over forced modes, for grids too large to
        synthesise whole."""
        nz, ny, nx = shape
        x = (i.to(torch.float64) + 0.5) / nx
        y = (j.to(torch.float64) + 0.5) / ny
        z = (k.to(torch.float64) + 0.5) / nz
        a = torch.zeros((3,) + tuple(k.shape), dtype=torch.float64)
        for m, (mx, my, mz) in enumerate(forced_modes()):
            e = torch.exp(1j * (2.0 * math.pi * (mx * x + my * y + mz * z)))
            for c in range(3):
                a[c] += 2.0 * (self.a_hat[m, c] * e).real
        return a * (self.a_rms / math.sqrt(self.mean_square()))


def apply_forcing(U: torch.Tensor, a: torch.Tensor, dt: float) -> torch.Tensor:
    """dm = rho a dt, dE = (m . a) dt, m before the kick (Sec. 3.1.1)."""
    out = U.clone()
    rho = U[0]
    out[1:4] = U[1:4] + rho * a * dt
    out[4] = U[4] + (U[1] * a[0] + U[2] * a[1] + U[3] * a[2]) * dt
    return out
