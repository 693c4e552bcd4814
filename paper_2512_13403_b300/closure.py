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
from .corrector import FORMS, Adam, Network, NPARAM, init_params, nparam
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
    # self-gravitating variant (Sec. 5.2): multigrid gravity, lognormal initial density of
    # this sigma (seeded per run), fluid at rest
    gravity: bool = False
    sigma: float = 1.0
    # coarse substeps per coarse interval: the coarse solver covers each interval with this many
    # equal steps; the pair's input is the state after all of them (the corrector is applied
    # once per interval, after the last)
    substeps: int = 1

    @property
    def coarse(self) -> int:
        return self.fine // self.factor


def _cfg(n, setup: ClosureSetup, seed):
    grav = dict(gravity=True, four_pi_G=1.0, mg_tol=1e-6, mg_max_cycles=30) if setup.gravity else {}
    return Config(shape=(n, n, n), precision="f32", forcing=setup.forcing, ou_seed=seed,
                  cooling=setup.cooling, t_floor=setup.t_floor, **grav)


def _initial_state(setup: ClosureSetup, n: int, seed: int) -> torch.Tensor:
    """The fine run's start: the driven cooling box (rho = 1, P = 0.6, at rest), or for the
    self-gravitating variant a lognormal density of the run's seed."""
    if setup.gravity:
        return inputs.self_gravitating_box_device((n, n, n), seed=seed, sigma=setup.sigma)
    return torch.from_numpy(inputs.cooling_box((n, n, n))).float().cuda().contiguous()


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
        fine.init_state(_initial_state(setup, n, setup.seed0 + r))
        fine.advance(setup.spinup_steps)
        for s in range(setup.snapshots):
            Uc0 = downsample(fine.get_state(), setup.factor)
            coarse.init_state(Uc0)
            dt_c = coarse.compute_dt()
            modes = fine_interval(fine, dt_c, setup.forcing)
            if modes is not None:
                coarse.set_forcing_modes(modes, hold=True)
            for _ in range(setup.substeps):
                coarse.step(dt_c / setup.substeps, sync=False)
            X[k] = coarse.get_state()
            Y[k] = downsample(fine.get_state(), setup.factor)
            k += 1
        if log:
            log(f"pairs: run {r + 1}/{setup.runs} done ({k} pairs)")
        fine.close()
    coarse.close()
    return X, Y


def normalisation(X: torch.Tensor, Y: torch.Tensor, net: Network):
    """Per-channel input mean/std and residual (Y - X) std, the correction's output scale
    (dh_cnn_field_moments on the network's grid)."""
    mu, sd = net.field_moments(X.contiguous())
    _, rsd = net.field_moments(Y.contiguous(), X.contiguous())
    return mu, [max(v, 1e-12) for v in sd], [max(v, 1e-12) for v in rsd]


def train(X: torch.Tensor, Y: torch.Tensor, epochs: int = 4, lr0: float = 1e-3, lr1: float = 1e-4,
          seed: int = 0, log=None, form: str = "state"):
    """Adam on the pair set, one pair per step, learning rate decayed geometrically from lr0 to
    lr1.  Returns (params, (mu, sigma, out_scale), losses)."""
    shape = tuple(X.shape[2:])
    net = Network(shape, form=form)
    mu, sigma, out = normalisation(X, Y, net)
    params = init_params(seed, out_scale=0.01, form=form).cuda()
    opt = Adam(params, lr=lr0)
    grads = torch.zeros(nparam(form), dtype=torch.float32, device="cuda")
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


def _set_corrector(solver: Solver, params, norm, form: str = "state"):
    import ctypes as C
    mu, sigma, out = norm
    normbuf = (C.c_float * 15)(*[float(v) for v in list(mu) + list(sigma) + list(out)])
    p = params.detach().float().cuda().contiguous()
    _lib.check(_lib.load().dh_set_corrector_form(solver.ctx, FORMS[form], C.c_void_p(p.data_ptr()),
                                                 normbuf), solver.ctx)


def _timed(fn) -> float:
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    fn()
    ev1.record()
    ev1.synchronize()
    return ev0.elapsed_time(ev1)


def equal_time_substeps(setup: ClosureSetup, params, norm, U0: torch.Tensor, probes: int = 10) -> int:
    """Substeps that give the uncorrected coarse run the GPU time of one corrected coarse step:
    round(t_corrected / t_uncorrected), measured on scratch runs from U0."""
    nc = setup.coarse
    plain = Solver(_cfg(nc, setup, 0))
    corr = Solver(_cfg(nc, setup, 0))
    plain.init_state(U0)
    corr.init_state(U0)
    _set_corrector(corr, params, norm)
    corr.correct_every_step(True)
    tp = tc = 0.0
    for k in range(probes + 2):
        dt = plain.compute_dt()
        a = _timed(lambda: plain.step(dt, sync=False))
        b = _timed(lambda: corr.step(dt, sync=False))
        if k >= 2:            # the first steps warm up the kernels
            tp += a
            tc += b
    plain.close()
    corr.close()
    return max(1, int(round(tc / tp)))


def evaluate(setup: ClosureSetup, params, norm, steps: int = 100, seeds=(200,),
             equal_time_substeps_n="auto", form: str = "state"):
    """Corrected and uncorrected coarse runs against the downsampled fine run, same forcing.

    For every held-out seed, a fine run is spun up and downsampled; coarse runs start from that
    state and advance one coarse step per fine interval (the table of the interval held, as in
    make_pairs).  A third run, uncorrected, takes `equal_time_substeps_n` substeps per coarse
    step: the uncorrected solver given the corrected run's GPU time as a smaller time step
    ("auto": from the measured cost ratio).  Returns (per-step relative L2 errors averaged over
    the seeds, GPU ms per coarse step of each run, the substep count).  A run whose state stops
    being finite ends there and counts as an infinite error afterwards; `evaluate.diverged`
    maps such runs to (seed, coarse step).
    """
    n, nc = setup.fine, setup.coarse
    err = {"uncorrected": np.zeros(steps), "corrected": np.zeros(steps),
           "uncorrected_equal_gpu_time": np.zeros(steps)}
    gpu_ms = {k: 0.0 for k in err}
    diverged = {}          # run name -> (seed, coarse step) of a non-finite state
    sub = equal_time_substeps_n
    for seed in seeds:
        fine = Solver(_cfg(n, setup, seed))
        fine.init_state(_initial_state(setup, n, seed))
        fine.advance(setup.spinup_steps)
        U0 = downsample(fine.get_state(), setup.factor)
        if sub == "auto":
            sub = equal_time_substeps(setup, params, norm, U0)
        runs = {}
        for name in err:
            runs[name] = Solver(_cfg(nc, setup, seed))
            runs[name].init_state(U0)
        _set_corrector(runs["corrected"], params, norm, form)
        runs["corrected"].correct_every_step(True)   # the step applies the corrector
        live = dict(runs)
        for k in range(steps):
            dt_c = runs["uncorrected"].compute_dt()
            modes = fine_interval(fine, dt_c, setup.forcing)
            for name, s in list(live.items()):
                if modes is not None:
                    s.set_forcing_modes(modes, hold=True)
                if name == "uncorrected_equal_gpu_time":
                    def adv(s=s):
                        for _ in range(sub):
                            s.step(dt_c / sub, sync=False)
                else:
                    def adv(s=s):
                        s.step(dt_c, sync=False)
                try:
                    gpu_ms[name] += _timed(adv)
                    s.time()   # settles the enqueued steps: raises if one failed
                except _lib.DhError:
                    # a non-finite state: the run stops and its error is infinite from here
                    diverged.setdefault(name, (seed, k))
                    del live[name]
            ref = downsample(fine.get_state(), setup.factor)
            for name in runs:
                e = _rel_l2(live[name].get_state(), ref) if name in live else float("inf")
                err[name][k] += e / len(seeds)
        for s in list(runs.values()) + [fine]:
            s.close()
    nrun = steps * len(seeds)
    evaluate.diverged = diverged
    return ({k: v.tolist() for k, v in err.items()}, {k: v / nrun for k, v in gpu_ms.items()}, sub)


def evaluate_substeps(setup: ClosureSetup, params, norm, steps: int = 100, seeds=(200,),
                      frontier=(1, 2, 3, 4, 6, 8), form: str = "state"):
    """The corrected coarse run with setup.substeps substeps per interval (the corrector applied
    once, after the last) against uncorrected runs with each substep count of `frontier`, all
    driven by the same fine run and forcing tables as evaluate().  The uncorrected runs trace the
    plain solver's error against its GPU time; the equal-time comparison takes the frontier run
    whose GPU time per interval is nearest the corrected run's, and the best frontier error at
    any cost is reported beside it.  Returns a dict of mean and final errors and GPU ms per
    interval of every run."""
    n, nc = setup.fine, setup.coarse
    names = [f"uncorrected_{m}" for m in frontier] + ["corrected"]
    subs = {f"uncorrected_{m}": m for m in frontier}
    subs["corrected"] = setup.substeps
    err = {k: np.zeros(steps) for k in names}
    per_seed = {k: {} for k in names}
    gpu_ms = {k: 0.0 for k in names}
    for seed in seeds:
        fine = Solver(_cfg(n, setup, seed))
        fine.init_state(_initial_state(setup, n, seed))
        fine.advance(setup.spinup_steps)
        U0 = downsample(fine.get_state(), setup.factor)
        runs = {k: Solver(_cfg(nc, setup, seed)) for k in names}
        for s in runs.values():
            s.init_state(U0)
        _set_corrector(runs["corrected"], params, norm, form)
        clock = Solver(_cfg(nc, setup, seed))   # single-step run whose CFL step sets the interval
        clock.init_state(U0)
        for k in range(steps):
            dt_c = clock.compute_dt()
            modes = fine_interval(fine, dt_c, setup.forcing)
            if modes is not None:
                clock.set_forcing_modes(modes, hold=True)
            clock.step(dt_c, sync=False)
            for name, s in runs.items():
                if modes is not None:
                    s.set_forcing_modes(modes, hold=True)
                m = subs[name]

                def adv(s=s, m=m, corr=name == "corrected"):
                    for j in range(m):
                        if corr:
                            s.correct_every_step(j == m - 1)
                        s.step(dt_c / m, sync=False)
                gpu_ms[name] += _timed(adv)
                s.time()
            ref = downsample(fine.get_state(), setup.factor)
            for name, s in runs.items():
                e = _rel_l2(s.get_state(), ref)
                err[name][k] += e / len(seeds)
                per_seed[name][seed] = per_seed[name].get(seed, 0.0) + e / steps
        for s in list(runs.values()) + [fine, clock]:
            s.close()
    nrun = steps * len(seeds)
    ms = {k: v / nrun for k, v in gpu_ms.items()}
    mean = {k: float(v.mean()) for k, v in err.items()}
    plain = [k for k in names if k != "corrected"]
    eq = min(plain, key=lambda k: abs(ms[k] - ms["corrected"]))
    best = min(plain, key=lambda k: mean[k])
    return {"substeps": setup.substeps, "mean_error": mean,
            "final_error": {k: float(v[-1]) for k, v in err.items()},
            "per_seed_mean_error": per_seed, "gpu_ms_per_interval": ms, "equal_gpu_time_run": eq,
            "uncorrected_equal_gpu_time": mean[eq], "corrected": mean["corrected"],
            "best_uncorrected": {"run": best, "error": mean[best], "gpu_ms": ms[best]}}


def evaluate_coarsened(fine: Solver, coarse_cfg: Config, factor: int, params, norm, fine_steps: int = 20,
                       form: str = "state"):
    """A trained corrector applied to a coarsened copy of a running fine simulation (the
    self-gravitating benchmark configuration: its 256^3-trained corrector at 4x coarsening).

    From the fine solver's current state, runs on the coarse grid start from D(U_f): uncorrected,
    corrected after every coarse step, and uncorrected with round(t_corrected / t_uncorrected)
    substeps per coarse step (the corrected run's GPU time, from the first interval's timings).
    Each coarse interval takes the uncorrected run's CFL step; the fine run covers the same time
    (its first substep draws the OU update, the rest hold it, and the coarse runs take that
    table), until it has taken `fine_steps` steps.  Returns per-interval relative L2 errors
    (mean over fields) against D(U_f), the GPU ms per coarse interval of each run, and the
    fine run's steps and GPU ms."""
    U0 = downsample(fine.get_state(), factor)
    runs = {k: Solver(coarse_cfg) for k in ("uncorrected", "corrected", "uncorrected_equal_gpu_time")}
    for s in runs.values():
        s.init_state(U0)
    _set_corrector(runs["corrected"], params, norm, form)
    runs["corrected"].correct_every_step(True)
    # warm-up of the coarse kernels and the network on a scratch context (first launches load
    # modules and set attributes), so that the first interval's timings are representative
    scratch = Solver(coarse_cfg)
    scratch.init_state(U0)
    _set_corrector(scratch, params, norm, form)
    scratch.correct_every_step(True)
    for _ in range(2):
        scratch.step(scratch.compute_dt())
    scratch.close()
    forcing = coarse_cfg.forcing
    err = {k: [] for k in runs}
    gpu_ms = {k: 0.0 for k in runs}
    fine_ms, intervals, sub = 0.0, 0, None
    n0 = fine.time()[1]
    while fine.time()[1] - n0 < fine_steps:
        dt_c = runs["uncorrected"].compute_dt()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        modes = fine_interval(fine, dt_c, forcing)
        e1.record()
        e1.synchronize()
        fine_ms += e0.elapsed_time(e1)
        for name, s in runs.items():
            if modes is not None:
                s.set_forcing_modes(modes, hold=True)
            if name == "uncorrected_equal_gpu_time":
                if sub is None:
                    sub = max(1, int(round(gpu_ms["corrected"] / max(gpu_ms["uncorrected"], 1e-9))))
                def adv(s=s):
                    for _ in range(sub):
                        s.step(dt_c / sub, sync=False)
            else:
                def adv(s=s):
                    s.step(dt_c, sync=False)
            gpu_ms[name] += _timed(adv)
        ref = downsample(fine.get_state(), factor)
        for name, s in runs.items():
            err[name].append(_rel_l2(s.get_state(), ref))
        intervals += 1
    for s in runs.values():
        s.close()
    return {"errors": err, "mean_error": {k: sum(v) / len(v) for k, v in err.items()},
            "gpu_ms_per_interval": {k: v / intervals for k, v in gpu_ms.items()},
            "equal_time_substeps": sub, "intervals": intervals,
            "fine_steps": fine.time()[1] - n0, "fine_gpu_ms": fine_ms}


# ---- solver-in-the-loop training (Sec. 7) ------------------------------------------------------
@dataclasses.dataclass
class Trajectory:
    """A reference rollout on the coarse grid: the start state, the time step, OU table and
    downsampled fine state after each coarse interval."""
    U0: torch.Tensor
    dts: List[float]
    modes: list
    targets: List[torch.Tensor]


def make_trajectories(setup: ClosureSetup, count: int, length: int, seed0: int = 300, log=None):
    """`count` reference rollouts of `length` coarse intervals, each from a spun-up fine run
    (intervals, time steps and OU tables as in make_pairs)."""
    n, nc = setup.fine, setup.coarse
    coarse = Solver(_cfg(nc, setup, seed0))
    out = []
    for r in range(count):
        fine = Solver(_cfg(n, setup, seed0 + r))
        fine.init_state(_initial_state(setup, n, seed0 + r))
        fine.advance(setup.spinup_steps)
        U0 = downsample(fine.get_state(), setup.factor)
        dts, modes, targets = [], [], []
        for _ in range(length):
            coarse.init_state(downsample(fine.get_state(), setup.factor))
            dt_c = coarse.compute_dt()
            modes.append(fine_interval(fine, dt_c, setup.forcing))
            dts.append(dt_c)
            targets.append(downsample(fine.get_state(), setup.factor))
        out.append(Trajectory(U0, dts, modes, targets))
        fine.close()
        if log:
            log(f"trajectories: {r + 1}/{count}")
    coarse.close()
    return out


class RolloutTrainer:
    """Loss and gradient of the rollout loss through the solver's hand adjoint and the network's
    VJP, for a coarse solver configuration and a network form."""

    def __init__(self, shape, cfg: Config, form: str = "state", rho_floor_frac: float = 1e-6,
                 substeps: int = 1):
        self.substeps = int(substeps)    # equal solver steps per coarse interval
        self.shape = tuple(shape)
        self.cfg = cfg
        self.form = form
        self.net = Network(self.shape, form=form)
        self.solver = Solver(cfg)
        self.grads = torch.zeros(nparam(form), dtype=torch.float32, device="cuda")
        self.rho_floor_frac = rho_floor_frac

    def close(self):
        self.net.close()
        self.solver.close()

    def _start(self, U, modes):
        self.solver.init_state(U)
        if modes is not None:
            self.solver.set_forcing_modes(modes, hold=True)

    def loss_and_grad(self, traj: Trajectory, params, norm, weights):
        """L = (1/S) sum_s mean(((U_s - T_s) / w)^2), U_s = C(H_s(U_{s-1})), H_s the solver's
        `substeps` equal steps over interval s; returns (L, dL/dparams).
        Every term and gradient is a library call: the loss terms and their gradients
        (dh_cnn_rollout_misfit), the floors (dh_cnn_floor_vjp), the network (dh_cnn_vjp), the
        solver step (dh_adjoint_advance_dt) and the sums (dh_axpy)."""
        from .corrector import axpy
        mu, sigma, out = norm
        self.net.set_params(params, mu, sigma, out)
        S = len(traj.dts)
        coef = 1.0 / (5 * traj.U0[0].numel() * S)
        rho_mean = self.net.field_moments(traj.U0.contiguous())[0][0]
        rho_floor = self.rho_floor_frac * rho_mean
        T_floor, gamma = self.cfg.t_floor, self.cfg.gamma
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        Us, Vs = [traj.U0], []
        for k in range(S):
            self._start(Us[-1], traj.modes[k])
            for _ in range(self.substeps):
                self.solver.step(traj.dts[k] / self.substeps, sync=False)
            V = self.solver.get_state()
            Vs.append(V)
            Un = V.clone()
            self.net.correct_state(Un, rho_floor, T_floor, gamma)
            Us.append(Un)
            self.net.rollout_misfit(Un, traj.targets[k], weights, coef, loss_acc=loss)
        total = torch.zeros_like(self.grads)
        lam = torch.empty_like(Us[S])
        self.net.rollout_misfit(Us[S], traj.targets[S - 1], weights, coef, lam=lam)
        for k in reversed(range(S)):
            self.net.forward(Vs[k])
            self.net.floor_vjp(Vs[k], lam, rho_floor, T_floor, gamma)
            gU = self.net.vjp(lam.contiguous(), self.grads)
            axpy(1.0, self.grads, total)
            axpy(1.0, lam, gU)                   # dL/dV = (I + J_dU)^T dL/dY
            self._start(Us[k], traj.modes[k])
            m = self.substeps
            lam = self.solver.adjoint_advance(m, m, gU, dt=traj.dts[k] / m)
            if k > 0:
                self.net.rollout_misfit(Us[k], traj.targets[k - 1], weights, coef, lam=lam,
                                        accumulate=True)
        return float(loss.item()), total


def train_rollout(trajs: List[Trajectory], setup: ClosureSetup, params, norm, iters: int,
                  lr: float = 1e-4, form: str = "state", weights=None, log=None):
    """Adam on the rollout loss, one trajectory per iteration (cycling).  Returns
    (params, losses, ms per iteration)."""
    nc = setup.coarse
    tr = RolloutTrainer((nc, nc, nc), _cfg(nc, setup, 0), form, substeps=setup.substeps)
    if weights is None:
        # the per-field spread of the targets (the paper weights fields to comparable ranges)
        allt = torch.stack([t for trj in trajs for t in trj.targets]).contiguous()
        weights = [max(v, 1e-12) for v in tr.net.field_moments(allt)[1]]
        del allt
    params = params.clone()
    opt = Adam(params, lr=lr)
    losses = []
    t0 = None
    for it in range(iters):
        if it == 1:                      # the first iteration loads kernels and allocates
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        L, g = tr.loss_and_grad(trajs[it % len(trajs)], params, norm, weights)
        opt.step(g)
        losses.append(L)
        if log and (it + 1) % max(1, iters // 10) == 0:
            log(f"rollout training: iteration {it + 1}/{iters} loss {L:.4e}")
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / max(iters - 1, 1) if t0 is not None else float("nan")
    tr.close()
    return params, losses, ms
