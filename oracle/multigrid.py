"""Oracle: multigrid Poisson solve for self-gravity (Sec. 5.2; App. C).  Test infrastructure only.

Solves A phi = F on a periodic grid with cubic cells of width h, where A is the seven-point
Laplacian (Sec. 5.2) and F = 4 pi G (rho - <rho>) (Sec. 5.1, mean-subtracted source).

Readings:
  * Smoothers: red-black Gauss-Seidel (default here) and weighted Jacobi (the paper's default,
    Sec. 5.2).  RBGS: red = (i+j+k) even, updated first, then black, each from the latest values:
    phi_i = (sum of 6 neighbours - h^2 F_i) / 6.  Jacobi: phi + omega D^{-1} (F - A phi) with
    D = -6/h^2, i.e. (1 - omega) phi + (omega/6)(sum of 6 neighbours - h^2 F), omega = 2/3.  The
    paper's component form prints the first coefficient as (1 - omega)/6; the matrix form it
    expands fixes it at (1 - omega), which is what is built.
  * Cycles (App. C): V visits each coarser level once; W visits the next coarser level twice
    (the second visit starting from the first's correction), recursively, except a coarsest level
    solved exactly, which is visited once (a second exact solve changes nothing).
  * Restriction: mean of the 8 children (Sec. 5.2 full-weighting formula with 1/8).
  * Prolongation: cell-centred trilinear interpolation from the 8 nearest coarse cells; per axis
    a fine cell takes 3/4 of its parent and 1/4 of the parent's neighbour on its side, giving the
    tensor-product weights (27, 9, 9, 9, 3, 3, 3, 1) / 64; periodic.
  * Coarse operator: the same seven-point Laplacian re-discretised with h_c = 2 h.
  * Levels: halve while every dimension is even and at least 8; the coarsest grid (at most 1024
    cells) is solved exactly with the pseudo-inverse of its dense operator, which also projects
    out the mean (the constant null space of the periodic problem).
  * Gauge and stopping: subtract <phi> after each cycle (<Phi> = 0, Sec. 5.1); stop when
    ||F - A phi||_2 / ||F||_2 <= tol (float64 norms) or after max_cycles; warm start from the
    caller's phi.
  * Force (Sec. 5): g_a = -(phi_{i+1} - phi_{i-1}) / (2 h); dm = rho g dt, dE = (m . g) dt with m
    taken before the kick.

Pins: tests/test_oracle_multigrid.py (single discrete Fourier mode against its exact discrete
solution F / lambda, FFT solve of the same operator, pseudo-inverse coarse solve, residual
reduction per cycle, restriction/prolongation identities on constants and linear fields; the
FFT solve itself against a single mode and against converged V-cycles).
"""
from __future__ import annotations

import math

import torch


def apply_A(phi: torch.Tensor, h: float) -> torch.Tensor:
    s = -6.0 * phi
    for d in range(3):
        s = s + torch.roll(phi, 1, dims=d) + torch.roll(phi, -1, dims=d)
    return s / (h * h)


def _color_masks(shape):
    nz, ny, nx = shape
    k = torch.arange(nz)[:, None, None]
    j = torch.arange(ny)[None, :, None]
    i = torch.arange(nx)[None, None, :]
    red = ((i + j + k) % 2) == 0
    return red, ~red


def rbgs_sweep(phi: torch.Tensor, F: torch.Tensor, h: float) -> torch.Tensor:
    """One red then black Gauss-Seidel pass."""
    red, black = _color_masks(phi.shape)
    for mask in (red, black):
        nb = torch.zeros_like(phi)
        for d in range(3):
            nb = nb + torch.roll(phi, 1, dims=d) + torch.roll(phi, -1, dims=d)
        phi = torch.where(mask, (nb - h * h * F) / 6.0, phi)
    return phi


def jacobi_sweep(phi: torch.Tensor, F: torch.Tensor, h: float, omega: float) -> torch.Tensor:
    """One weighted Jacobi pass: phi + omega D^{-1} (F - A phi), D = -6/h^2 (Sec. 5.2)."""
    return phi + omega * (-(h * h) / 6.0) * (F - apply_A(phi, h))


def restrict(r: torch.Tensor) -> torch.Tensor:
    nz, ny, nx = r.shape
    return r.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(dim=(1, 3, 5))


def _prolong_axis(e: torch.Tensor, d: int) -> torch.Tensor:
    prev = torch.roll(e, 1, dims=d)
    nxt = torch.roll(e, -1, dims=d)
    even = 0.75 * e + 0.25 * prev
    odd = 0.75 * e + 0.25 * nxt
    out = torch.stack([even, odd], dim=d + 1)
    shape = list(e.shape)
    shape[d] *= 2
    return out.reshape(shape)


def prolong(e: torch.Tensor) -> torch.Tensor:
    for d in range(3):
        e = _prolong_axis(e, d)
    return e


def level_shapes(shape):
    shapes = [tuple(shape)]
    while all(n % 2 == 0 and n >= 8 for n in shapes[-1]):
        shapes.append(tuple(n // 2 for n in shapes[-1]))
    if math.prod(shapes[-1]) > 1024:
        raise ValueError(f"coarsest multigrid level {shapes[-1]} exceeds 1024 cells")
    return shapes


def dense_operator(shape, h: float) -> torch.Tensor:
    n = math.prod(shape)
    A = torch.zeros(n, n, dtype=torch.float64)
    eye = torch.eye(n, dtype=torch.float64).reshape((n,) + tuple(shape))
    for col in range(n):
        A[:, col] = apply_A(eye[col], h).reshape(-1)
    return A


_PINV_CACHE = {}


def coarse_solve(F: torch.Tensor, h: float) -> torch.Tensor:
    key = (tuple(F.shape), h)
    if key not in _PINV_CACHE:
        _PINV_CACHE[key] = torch.linalg.pinv(dense_operator(F.shape, h))
    return (_PINV_CACHE[key] @ F.reshape(-1)).reshape(F.shape)


def cycle(phi, F, h, shapes, level=0, npre=2, npost=2, smoother="rbgs", omega=2.0 / 3.0, gamma=1):
    """One multigrid cycle on A phi = F: gamma = 1 is the V-cycle, gamma = 2 the W-cycle."""
    if level == len(shapes) - 1:
        return coarse_solve(F, h)

    def smooth(p):
        return rbgs_sweep(p, F, h) if smoother == "rbgs" else jacobi_sweep(p, F, h, omega)

    for _ in range(npre):
        phi = smooth(phi)
    rc = restrict(F - apply_A(phi, h))
    ec = torch.zeros_like(rc)
    visits = gamma if level + 1 < len(shapes) - 1 else 1
    for _ in range(visits):
        ec = cycle(ec, rc, 2.0 * h, shapes, level + 1, npre, npost, smoother, omega, gamma)
    phi = phi + prolong(ec)
    for _ in range(npost):
        phi = smooth(phi)
    return phi


def vcycle(phi, F, h, shapes, level=0, npre=2, npost=2):
    return cycle(phi, F, h, shapes, level, npre, npost)


def relative_residual(phi, F, h) -> float:
    nF = float(torch.linalg.vector_norm(F))
    if nF == 0.0:
        return 0.0
    return float(torch.linalg.vector_norm(F - apply_A(phi, h))) / nF


def solve(F: torch.Tensor, h: float, phi0=None, tol=1e-6, max_cycles=30, npre=2, npost=2,
          smoother="rbgs", omega=2.0 / 3.0, cycle_type="V"):
    """Cycles until the relative residual meets tol; returns (phi, cycles, rel_res, converged)."""
    shapes = level_shapes(F.shape)
    phi = torch.zeros_like(F) if phi0 is None else phi0.clone()
    if float(torch.linalg.vector_norm(F)) == 0.0:
        return torch.zeros_like(F), 0, 0.0, True
    res = relative_residual(phi, F, h)
    cycles = 0
    while res > tol and cycles < max_cycles:
        phi = cycle(phi, F, h, shapes, 0, npre, npost, smoother, omega, 2 if cycle_type == "W" else 1)
        phi = phi - phi.mean()
        cycles += 1
        res = relative_residual(phi, F, h)
    return phi, cycles, res, res <= tol


def fft_solve(F: torch.Tensor, h: float) -> torch.Tensor:
    """Exact A phi = F - <F>, <phi> = 0, for the same seven-point operator: on a periodic grid
    the DFT diagonalises A, with eigenvalue -(4/h^2) sum_a sin^2(pi k_a / n_a) for mode k.  A
    plain library FFT, differentiable; the reference the multigrid iterates converge to."""
    nz, ny, nx = F.shape
    s = lambda n: torch.sin(math.pi * torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64) / n) ** 2
    lam = -(4.0 / h ** 2) * (s(nz)[:, None, None] + s(ny)[None, :, None] + s(nx)[None, None, :])
    keep = torch.ones_like(lam)
    keep[0, 0, 0] = 0.0
    lam = torch.where(keep > 0, lam, torch.ones_like(lam))
    return torch.fft.ifftn(torch.fft.fftn(F) * keep / lam).real


def poisson_source(rho: torch.Tensor, four_pi_G: float) -> torch.Tensor:
    return four_pi_G * (rho - rho.mean())


def gravity_source(U: torch.Tensor, phi: torch.Tensor, dt: float, h: float) -> torch.Tensor:
    out = U.clone()
    rho = U[0]
    g = [-(torch.roll(phi, -1, dims=2 - a) - torch.roll(phi, 1, dims=2 - a)) / (2.0 * h)
         for a in range(3)]
    for a in range(3):
        out[1 + a] = U[1 + a] + rho * g[a] * dt
    out[4] = U[4] + (U[1] * g[0] + U[2] * g[1] + U[3] * g[2]) * dt
    return out
