"""Learned closure for the coarse solver: training pairs made by the solver itself, training of
the residual corrector, and its evaluation against a downsampled fine run.

All numerical work runs in libdh.so (solver steps, the 4^3 block mean, the tensor-core network
and its training step, Adam); this module sequences the calls and reports error norms.

Pairs (one per coarse step of a fine run): input = one coarse step H_c applied to D4 U_f(t),
target = D4 U_f(t + dt_c), with D4 the 4^3 block mean of the conserved fields and the fine run
landing exactly on t + dt_c (its last step clipped).  Forcing: over each coarse interval the
fine run draws and applies one OU update in its first substep and then holds that table for its
remaining substeps, and the coarse step is driven with the same table; both grids thus see one
acceleration history, and the pair isolates the coarse discretisation error instead of the
difference between two noise realisations.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import List

import numpy as np
import torch

from . import _lib, inputs
from .corrector import Adam, Network, NPARAM, init_params
from .solver import Config, Solver


@dataclasses.dataclass
class ClosureSetup:
    fine: int = 256
    factor: int = 4
    runs: int = 20
    snapshots: int = 100
    spinup_steps: int = 200
    seed0: int = 100
    forcing: bool = True
    cooling: bool = True
    t_floor: float = 0.05

    @property
    def coarse(self) -> int:
        return self.fine // self.factor


def _cfg(n, setup: ClosureSetup, seed):
    return Config(shape=(n, n, n), precision="f32", forcing=setup.forcing, ou_seed=seed,
                  cooling=setup.cooling, t_floor=setup.t_floor)


def downsample(Uf: torch.Tensor, factor: int) -> torch.Tensor:
    lib = _lib.load()
    nz, ny, nx = Uf.shape[1:]
    Uc = torch.empty((5, nz // factor, ny // factor, nx // factor), dtype=torch.float32, device="cuda")
    st = lib.dh_downsample(Uf.data_ptr(), nx, ny, nz, factor, Uc.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    _lib.check(st)
    return Uc


def advance_to(solver: Solver, dt_total: float):
    """Advance by exactly dt_total with CFL steps, the last one clipped."""
    t = 0.0
    while dt_total - t > 1e-14 * max(1.0, dt_total):
        dt = min(solver.compute_dt(), dt_total - t)
        solver.step(dt)
        t += dt


def fine_interval(fine: Solver, dt_c: float, forcing: bool):
    """Advance the fine run by dt_c: the first substep takes a fresh OU update, the rest hold the
    table.  Returns the table of the interval (None without forcing)."""
    if forcing:
        fine.set_forcing_modes(fine.forcing_modes(), hold=False)
    dt1 = min(fine.compute_dt(), dt_c)
    fine.step(dt1)
    modes = None
    if forcing:
        modes = fine.forcing_modes()
        fine.set_forcing_modes(modes, hold=True)
    advance_to(fine, dt_c - dt1)
    return modes


def make_pairs(setup: ClosureSetup, log=None):
    """Returns (inputs, targets): float32 CUDA tensors of shape (P, 5, n, n, n)."""
    n, nc = setup.fine, setup.coarse
    P = setup.runs * setup.snapshots
    X = torch.empty((P, 5, nc, nc, nc), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    coarse = Solver(_cfg(nc, setup, setup.seed0))
    k = 0
    for r in range(setup.runs):
        fine = Solver(_cfg(n, setup, setup.seed0 + r))
        fine.init_state(torch.from_numpy(inputs.cooling_box((n, n, n))).float().cuda().contiguous())
        fine.advance(setup.spinup_steps)
        for s in range(setup.snapshots):
            Uc0 = downsample(fine.get_state(), setup.factor)
            coarse.init_state(Uc0)
            dt_c = coarse.compute_dt()
            modes = fine_interval(fine, dt_c, setup.forcing)
            if modes is not None:
                coarse.set_forcing_modes(modes, hold=True)
            coarse.step(dt_c)
            X[k] = coarse.get_state()
            Y[k] = downsample(fine.get_state(), setup.factor)
            k += 1
        if log:
            log(f"pairs: run {r + 1}/{setup.runs} done ({k} pairs)")
        fine.close()
    coarse.close()
    return X, Y


def normalisation(X: torch.Tensor, Y: torch.Tensor):
    """Per-channel input mean/std and residual std (the correction's output scale)."""
    mu = [float(X[:, c].mean()) for c in range(5)]
    sigma = [max(float(X[:, c].std()), 1e-12) for c in range(5)]
    R = Y - X
    out = [max(float(R[:, c].std()), 1e-12) for c in range(5)]
    return mu, sigma, out


def train(X: torch.Tensor, Y: torch.Tensor, epochs: int = 4, lr0: float = 1e-3, lr1: float = 1e-4,
          seed: int = 0, log=None):
    """Adam on the pair set, one pair per step, learning rate decayed geometrically from lr0 to
    lr1.  Returns (params, (mu, sigma, out_scale), losses)."""
    shape = tuple(X.shape[2:])
    net = Network(shape)
    mu, sigma, out = normalisation(X, Y)
    params = init_params(seed, out_scale=0.01).cuda()
    opt = Adam(params, lr=lr0)
    grads = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
    g = np.random.default_rng(seed)
    P = X.shape[0]
    total = epochs * P
    losses = []
    it = 0
    for ep in range(epochs):
        perm = g.permutation(P)
        acc = 0.0
        for i in perm:
            opt.lr = lr0 * (lr1 / lr0) ** (it / max(total - 1, 1))
            net.set_params(params, mu, sigma, out)
            net.forward(X[i])
            acc += net.backward(X[i], Y[i], grads)
            opt.step(grads)
            it += 1
        losses.append(acc / P)
        if log:
            log(f"train: epoch {ep + 1}/{epochs} mean loss {losses[-1]:.4e}")
    net.close()
    return params, (mu, sigma, out), losses


def _rel_l2(U: torch.Tensor, R: torch.Tensor) -> float:
    """Mean over the five fields of ||U_f - R_f|| / ||R_f||."""
    return float(sum(float(torch.linalg.vector_norm(U[c] - R[c]) / torch.linalg.vector_norm(R[c]))
                     for c in range(5)) / 5.0)


def evaluate(setup: ClosureSetup, params, norm, steps: int = 100, seed: int = 200,
             equal_time_substeps: int = 0):
    """Corrected and uncorrected coarse runs against the downsampled fine run, same forcing.

    Returns per-step relative L2 errors and the GPU time per coarse step of each run.  With
    equal_time_substeps > 1 a third run, uncorrected, takes that many substeps per coarse step
    (the uncorrected solver given the corrected run's GPU time as a smaller time step).
    """
    n, nc = setup.fine, setup.coarse
    fine = Solver(_cfg(n, setup, seed))
    fine.init_state(torch.from_numpy(inputs.cooling_box((n, n, n))).float().cuda().contiguous())
    fine.advance(setup.spinup_steps)
    U0 = downsample(fine.get_state(), setup.factor)
    plain = Solver(_cfg(nc, setup, seed))
    corr = Solver(_cfg(nc, setup, seed))
    plain.init_state(U0)
    corr.init_state(U0)
    mu, sigma, out = norm
    import ctypes as C
    normbuf = (C.c_float * 15)(*[float(v) for v in list(mu) + list(sigma) + list(out)])
    p = params.detach().float().cuda().contiguous()
    _lib.check(_lib.load().dh_set_corrector(corr.ctx, C.c_void_p(p.data_ptr()), normbuf), corr.ctx)
    runs = {"uncorrected": plain, "corrected": corr}
    if equal_time_substeps > 1:
        eq = Solver(_cfg(nc, setup, seed))
        eq.init_state(U0)
        runs["uncorrected_equal_gpu_time"] = eq
    err = {k: [] for k in runs}
    gpu_ms = {k: 0.0 for k in runs}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(steps):
        dt_c = plain.compute_dt()
        modes = fine_interval(fine, dt_c, setup.forcing)
        for s in runs.values():
            if modes is not None:
                s.set_forcing_modes(modes, hold=True)
        for name, s in runs.items():
            ev0.record()
            if name == "uncorrected_equal_gpu_time":
                for _ in range(equal_time_substeps):
                    s.step(dt_c / equal_time_substeps, sync=False)
            else:
                s.step(dt_c, sync=False)
            if name == "corrected":
                _lib.check(_lib.load().dh_correct(s.ctx), s.ctx)
            ev1.record()
            ev1.synchronize()
            gpu_ms[name] += ev0.elapsed_time(ev1)
        ref = downsample(fine.get_state(), setup.factor)
        for name, s in runs.items():
            err[name].append(_rel_l2(s.get_state(), ref))
    for s in list(runs.values()) + [fine]:
        s.close()
    return err, {k: v / steps for k, v in gpu_ms.items()}
