"""Seeded synthetic inputs: initial conditions for the periodic Euler solver.

This module only builds input states (and the random draws that define them).  It holds none
of the solver's update arithmetic and imports neither the CUDA binding nor the CPU oracle, so
both sides can be fed the very same bits.

Layout of every state returned here: a float64 numpy array ``U`` of shape ``(5, nz, ny, nx)``
holding the conserved fields ``(rho, m_x, m_y, m_z, E)`` of the paper's Eq. 2, x fastest, so
that ``U.reshape(5, -1)`` is the structure-of-arrays layout the library expects.

Recipes (paper sections in brackets):
  * ``kelvin_helmholtz``: the shear layer used for the Kelvin-Helmholtz comparison (App. B.2),
    here as a 3D slab: rho=2, vx=-0.5 inside |y-0.5|<0.25, rho=1, vx=+0.5 outside, P=2.5,
    vy uniform in [-0.01, 0.01) from a seeded generator, vz=0, no interface smoothing.
  * ``gaussian_field``: Hermitian Gaussian random field with |g_k|^2 ~ k^p over the integer
    modes 1 <= |n| < N/2 (Sec. 3.1, Eq. for A(k) ~ k^(p/2)), scaled to unit variance.
  * ``lognormal_density``: rho = exp(sigma g) / <exp(sigma g)>, g from a k^-2 field.
  * ``turbulent_velocity``: three independent k^-4 Gaussian components (unprojected), rescaled
    to a target rms Mach number with the local sound speed (Sec. 3.1, Eq. for alpha).
  * ``decaying_turbulence``, ``cooling_box``, ``self_gravitating_box``: the three turbulence
    set-ups, assembled conservatively as in Sec. 3.1 (rho, m = rho u, E = P/(gamma-1) + rho u^2/2).
  * ``sound_wave``, ``double_sod``: smooth and discontinuous 1D-in-x states for convergence
    and exact-Riemann checks.
"""
from __future__ import annotations

import numpy as np


def prim_to_state(rho, vx, vy, vz, P, gamma):
    """Assemble conserved fields from primitive ones (Sec. 3.1 conservative initialisation)."""
    rho = np.asarray(rho, dtype=np.float64)
    U = np.empty((5,) + rho.shape, dtype=np.float64)
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = P / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return U


def _centres(n):
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def uniform_state(shape, rho=1.0, P=0.6, v=(0.0, 0.0, 0.0), gamma=5.0 / 3.0):
    nz, ny, nx = shape
    z = np.zeros(shape)
    return prim_to_state(z + rho, z + v[0], z + v[1], z + v[2], z + P, gamma)


def kelvin_helmholtz(shape, seed=0, gamma=5.0 / 3.0, amp=0.01):
    """Shear layer on the unit periodic box; shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    y = _centres(ny)[None, :, None] * np.ones(shape)
    inside = np.abs(y - 0.5) < 0.25
    rho = np.where(inside, 2.0, 1.0)
    vx = np.where(inside, -0.5, 0.5)
    rng = np.random.default_rng(seed)
    vy = amp * 2.0 * (rng.random(shape) - 0.5)
    vz = np.zeros(shape)
    P = np.full(shape, 2.5)
    return prim_to_state(rho, vx, vy, vz, P, gamma)


def _wavenumber_magnitude(shape):
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    return np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)


def gaussian_field(shape, p, seed):
    """Unit-variance Gaussian random field with power |g_k|^2 ~ |n|^p on 1 <= |n| < min(N)/2.

    White noise is drawn in real space (so the spectrum is Hermitian by construction),
    transformed, multiplied by A(k) = |n|^(p/2) inside the band and zero outside, and
    transformed back.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    kmag = _wavenumber_magnitude(shape)
    band = (kmag >= 1.0) & (kmag < min(shape) / 2.0)
    amp = np.zeros(shape)
    amp[band] = kmag[band] ** (p / 2.0)
    g = np.fft.ifftn(np.fft.fftn(noise) * amp).real
    g -= g.mean()
    return g / g.std()


def lognormal_density(shape, sigma, seed):
    g = gaussian_field(shape, -2.0, seed)
    e = np.exp(sigma * g)
    return e / e.mean()


def turbulent_velocity(shape, seed, mach, rho, P, gamma, p=-4.0):
    """Three independent k^p components, rescaled so that rms|u| = mach * <c_s> (Sec. 3.1)."""
    comps = [gaussian_field(shape, p, seed * 7919 + 101 + c) for c in range(3)]
    u = np.stack(comps)
    cs = np.sqrt(gamma * P / rho)
    alpha = mach * cs.mean() / np.sqrt((u * u).sum(0).mean())
    return alpha * u


def decaying_turbulence(shape, seed=2, sigma=0.5, mach=2.0, P0=0.6, gamma=5.0 / 3.0, p_sigma=0.0):
    """Lognormal density, k^-4 velocities at rms Mach `mach`, pressure P0.  p_sigma > 0 adds
    lognormal pressure fluctuations (a generic state: no exactly uniform field)."""
    rho = lognormal_density(shape, sigma, seed)
    P = np.full(shape, P0) if p_sigma == 0.0 else P0 * lognormal_density(shape, p_sigma, seed + 977)
    u = turbulent_velocity(shape, seed, mach, rho, P, gamma)
    return prim_to_state(rho, u[0], u[1], u[2], P, gamma)


def cooling_box(shape, rho0=1.0, P0=0.6, gamma=5.0 / 3.0):
    return uniform_state(shape, rho=rho0, P=P0, gamma=gamma)


def self_gravitating_box(shape, seed=5, sigma=1.0, P0=0.6, gamma=5.0 / 3.0):
    rho = lognormal_density(shape, sigma, seed)
    z = np.zeros(shape)
    return prim_to_state(rho, z, z, z, z + P0, gamma)


def sound_wave(nx, ny=4, nz=4, amp=1e-6, rho0=1.0, P0=1.0 / 1.4, gamma=1.4):
    """Right-moving linear acoustic wave along x with one wavelength in the box."""
    shape = (nz, ny, nx)
    x = _centres(nx)[None, None, :] * np.ones(shape)
    c0 = np.sqrt(gamma * P0 / rho0)
    s = amp * np.sin(2.0 * np.pi * x)
    rho = rho0 * (1.0 + s)
    vx = c0 * s
    P = P0 * (1.0 + gamma * s)
    z = np.zeros(shape)
    return prim_to_state(rho, vx, z, z, P, gamma)


def double_sod(nx, ny=4, nz=4, gamma=1.4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Sod states mirrored about x=0.5 so the periodic box holds two back-to-back tubes.

    Left state on 0.25 <= x < 0.75, right state elsewhere; interfaces at x=0.25 and x=0.75.
    """
    shape = (nz, ny, nx)
    x = _centres(nx)[None, None, :] * np.ones(shape)
    inner = (x >= 0.25) & (x < 0.75)
    rho = np.where(inner, left[0], right[0])
    vx = np.where(inner, left[1], right[1])
    P = np.where(inner, left[2], right[2])
    z = np.zeros(shape)
    return prim_to_state(rho, vx, z, z, P, gamma)


def lognormal_density_device(shape, sigma, seed, device="cuda"):
    """lognormal_density's recipe on the GPU in float32 for grids too large for the host
    (1024^3): white noise from torch's seeded generator (not numpy's stream), the |n|^-1
    amplitude (power |n|^-2) on 1 <= |n| < min(N)/2 through a real FFT, unit variance,
    rho = exp(sigma g) / <exp(sigma g)>."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    nz, ny, nx = shape
    F = torch.fft.rfftn(torch.randn(shape, generator=gen, device=device, dtype=torch.float32))
    kz = torch.fft.fftfreq(nz, d=1.0 / nz, device=device)
    ky = torch.fft.fftfreq(ny, d=1.0 / ny, device=device)
    kx = torch.fft.rfftfreq(nx, d=1.0 / nx, device=device)
    kmag = torch.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    band = (kmag >= 1.0) & (kmag < min(shape) / 2.0)
    F *= torch.where(band, kmag.clamp(min=1.0) ** -1.0, torch.zeros_like(kmag))
    del kmag, band
    g = torch.fft.irfftn(F, s=shape)
    del F
    g -= g.double().mean().float()
    g /= g.double().pow(2).mean().sqrt().float()
    e = torch.exp(sigma * g)
    del g
    return e / e.double().mean().float()


def self_gravitating_box_device(shape, seed=5, sigma=1.0, P0=0.6, gamma=5.0 / 3.0, device="cuda"):
    """self_gravitating_box on the GPU (float32 state, 5 planes): lognormal density from
    lognormal_density_device, fluid at rest, pressure P0."""
    import torch
    U = torch.zeros((5,) + tuple(shape), dtype=torch.float32, device=device)
    U[0] = lognormal_density_device(shape, sigma, seed, device)
    U[4] = P0 / (gamma - 1.0)
    return U
