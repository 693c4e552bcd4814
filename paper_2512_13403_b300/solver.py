"""Python face of the C ABI: a context wrapper that marshals torch tensors / numpy arrays.

No numerical work happens here; each method is one call into libdh.so (include/dh.h).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import DhConfig, check


@dataclasses.dataclass
class Config:
    """Mirror of dh_config (include/dh.h); shape is (nz, ny, nx)."""
    shape: tuple
    precision: str = "f32"
    dx: Optional[tuple] = None
    gamma: float = 5.0 / 3.0
    cfl: float = 0.4
    dt_max: float = math.inf
    forcing: bool = False
    ou_tau: float = 0.5
    ou_arms: float = 1.0
    ou_seed: int = 1
    cooling: bool = False
    t_floor: float = 0.05
    cool_frac: float = 0.1
    nsub_max: int = 1024
    gravity: bool = False
    four_pi_G: float = 1.0
    mg_tol: float = 1e-6
    mg_max_cycles: int = 30
    mg_pre: int = 2
    mg_post: int = 2
    mg_smoother: str = "rbgs"     # "rbgs" or "jacobi"
    mg_omega: float = 2.0 / 3.0
    mg_cycle: str = "V"           # "V" or "W"
    limiter: str = "mc"           # "mc" or "vanleer"
    integrator: str = "rk2"       # "rk2" or "ssprk3"
    c_cool: float = math.inf      # cooling time-step factor (Sec. 4.3); inf: off

    def to_c(self) -> DhConfig:
        nz, ny, nx = self.shape
        c = DhConfig()
        _lib.load().dh_config_default(C.byref(c), nx, ny, nz)
        c.precision = _lib.DH_F64 if self.precision == "f64" else _lib.DH_F32
        if self.dx is not None:
            c.dx, c.dy, c.dz = self.dx
        for f in ("gamma", "cfl", "dt_max", "ou_tau", "ou_arms", "t_floor", "cool_frac",
                  "four_pi_G", "mg_tol", "c_cool"):
            setattr(c, f, float(getattr(self, f)))
        for f in ("nsub_max", "mg_max_cycles", "mg_pre", "mg_post"):
            setattr(c, f, int(getattr(self, f)))
        c.forcing, c.cooling, c.gravity = int(self.forcing), int(self.cooling), int(self.gravity)
        c.mg_smoother = {"rbgs": 0, "jacobi": 1}[self.mg_smoother]
        c.mg_omega = float(self.mg_omega)
        c.mg_cycle = {"V": 1, "W": 2}[self.mg_cycle]
        c.limiter = {"mc": 0, "vanleer": 1}[self.limiter]
        c.integrator = {"rk2": 2, "ssprk3": 3}[self.integrator]
        c.ou_seed = int(self.ou_seed)
        return c


class Solver:
    """One dh_ctx on the current CUDA device and stream."""

    def __init__(self, cfg: Config, stream: Optional[torch.cuda.Stream] = None):
        self.lib = _lib.load()
        self.cfg = cfg
        self.dtype = torch.float64 if cfg.precision == "f64" else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ccfg = cfg.to_c()
        ctx = C.c_void_p()
        check(self.lib.dh_create(C.byref(ccfg), C.c_void_p(self.stream.cuda_stream), C.byref(ctx)))
        self.ctx = ctx
        self.shape = tuple(cfg.shape)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        check(status, self.ctx)

    def _as_buffer(self, x, nfield=5):
        """(pointer, on_device, keepalive) for a state-shaped array of the context dtype."""
        shape = (nfield,) + self.shape
        if isinstance(x, torch.Tensor):
            if tuple(x.shape) != shape or x.dtype != self.dtype or not x.is_contiguous():
                raise ValueError(f"expected contiguous {self.dtype} tensor of shape {shape}")
            return x.data_ptr(), int(x.is_cuda), x
        a = np.ascontiguousarray(x, dtype=np.float64 if self.dtype == torch.float64 else np.float32)
        if a.shape != shape:
            raise ValueError(f"expected array of shape {shape}")
        return a.ctypes.data, 0, a

    def init_state(self, U):
        ptr, dev, keep = self._as_buffer(U)
        if dev:
            torch.cuda.current_stream().synchronize()
        self._check(self.lib.dh_init_state(self.ctx, C.c_void_p(ptr), dev))

    def get_state(self, out=None, device=True):
        if out is None:
            out = torch.empty((5,) + self.shape, dtype=self.dtype,
                              device="cuda" if device else "cpu",
                              pin_memory=False)
        ptr, dev, keep = self._as_buffer(out)
        self._check(self.lib.dh_get_state(self.ctx, C.c_void_p(ptr), dev))
        return out

    def step(self, dt: float = 0.0, sync: bool = True) -> Optional[float]:
        if sync:
            d = C.c_double()
            self._check(self.lib.dh_step(self.ctx, float(dt), C.byref(d)))
            return d.value
        self._check(self.lib.dh_step(self.ctx, float(dt), None))
        return None

    def advance(self, n: int) -> float:
        t = C.c_double()
        self._check(self.lib.dh_advance(self.ctx, int(n), C.byref(t)))
        return t.value

    def time(self):
        t = C.c_double()
        n = C.c_longlong()
        self._check(self.lib.dh_get_time(self.ctx, C.byref(t), C.byref(n)))
        return t.value, n.value

    def compute_dt(self) -> float:
        d = C.c_double()
        self._check(self.lib.dh_compute_dt(self.ctx, C.byref(d)))
        return d.value

    def conserved_totals(self):
        out = (C.c_double * 5)()
        self._check(self.lib.dh_conserved_totals(self.ctx, out))
        return list(out)

    def metrics(self) -> dict:
        """The diagnostics record (dh_get_metrics): t, dt, nstep, flags, cool_max_substeps,
        slope_fallbacks, mg_cycles, mg_residual, totals, rho_min, p_min."""
        m = _lib.DhMetrics()
        self._check(self.lib.dh_get_metrics(self.ctx, C.byref(m)))
        return {"t": m.t, "dt": m.dt, "nstep": m.nstep, "flags": m.flags,
                "cool_max_substeps": m.cool_max_substeps, "slope_fallbacks": m.slope_fallbacks,
                "mg_cycles": m.mg_cycles,
                "mg_residual": m.mg_residual, "totals": list(m.totals), "rho_min": m.rho_min,
                "p_min": m.p_min}

    def forcing_field(self, device=True):
        out = torch.empty((3,) + self.shape, dtype=self.dtype, device="cuda" if device else "cpu")
        ptr, dev, keep = self._as_buffer(out, 3)
        self._check(self.lib.dh_forcing_field(self.ctx, C.c_void_p(ptr), dev))
        return out

    def forcing_modes(self) -> np.ndarray:
        out = (C.c_double * 96)()
        self._check(self.lib.dh_forcing_modes(self.ctx, out))
        a = np.frombuffer(out, dtype=np.float64).reshape(16, 3, 2)
        return a[..., 0] + 1j * a[..., 1]

    def set_forcing_modes(self, modes: np.ndarray, hold: bool):
        a = np.zeros((16, 3, 2), dtype=np.float64)
        a[..., 0] = np.real(modes)
        a[..., 1] = np.imag(modes)
        buf = (C.c_double * 96)(*a.reshape(-1).tolist())
        self._check(self.lib.dh_set_forcing_modes(self.ctx, buf, int(hold)))

    def potential(self):
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        cyc = C.c_int()
        res = C.c_double()
        self._check(self.lib.dh_get_potential(self.ctx, C.c_void_p(out.data_ptr()), 1,
                                              C.byref(cyc), C.byref(res)))
        return out, cyc.value, res.value

    def mg_stats(self):
        """(V-cycles, final relative residual) of the last Poisson solve."""
        cyc = C.c_int()
        res = C.c_double()
        self._check(self.lib.dh_get_potential(self.ctx, None, 1, C.byref(cyc), C.byref(res)))
        return cyc.value, res.value

    def fft_poisson(self, rho):
        """Exact Poisson solve by the DFT for one density plane (power-of-two grids); returns
        phi (float64, on the device)."""
        if not (isinstance(rho, torch.Tensor) and rho.is_cuda and rho.dtype == self.dtype
                and tuple(rho.shape) == self.shape and rho.is_contiguous()):
            raise ValueError("rho must be a contiguous device plane of the solver dtype")
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        self._check(self.lib.dh_fft_poisson(self.ctx, C.c_void_p(rho.data_ptr()), 1,
                                            C.c_void_p(out.data_ptr()), 1))
        return out

    def reset_potential(self):
        """Zero potential: the next solve starts cold."""
        self._check(self.lib.dh_reset_potential(self.ctx))

    def solve_poisson(self, rho, fetch: bool = True):
        """Standalone multigrid solve for one density plane; returns (phi, cycles, rel_res), or
        (None, cycles, rel_res) without fetch (phi stays in the context)."""
        if isinstance(rho, torch.Tensor):
            if rho.dtype != self.dtype or tuple(rho.shape) != self.shape or not rho.is_contiguous():
                raise ValueError("rho must be a contiguous plane of the solver dtype")
            ptr, dev, keep = rho.data_ptr(), int(rho.is_cuda), rho
        else:
            keep = np.ascontiguousarray(rho, dtype=np.float64 if self.dtype == torch.float64 else np.float32)
            ptr, dev = keep.ctypes.data, 0
        self._check(self.lib.dh_solve_poisson(self.ctx, C.c_void_p(ptr), dev))
        if not fetch:
            return (None,) + tuple(self.mg_stats())
        return self.potential()

    def adjoint_advance(self, n_steps: int, ckpt_every: int, dLdU_final, dt: float = 0.0):
        """dL/dU of the current state for n_steps steps (CFL steps, or each at dt > 0) and the
        gradient dLdU_final of the state they reach; the state itself advances."""
        ptr, dev, keep = self._as_buffer(dLdU_final)
        out = torch.empty((5,) + self.shape, dtype=self.dtype, device="cuda" if dev else "cpu")
        optr, odev, okeep = self._as_buffer(out)
        self._check(self.lib.dh_adjoint_advance_dt(self.ctx, int(n_steps), int(ckpt_every), float(dt),
                                                   C.c_void_p(ptr), C.c_void_p(optr), dev))
        return out

    def save(self, path: str):
        """File checkpoint (state, time, step count, OU tables, gravity warm start)."""
        self._check(self.lib.dh_save(self.ctx, str(path).encode()))

    def load(self, path: str):
        """Restore a checkpoint written by a context of the same configuration."""
        self._check(self.lib.dh_load(self.ctx, str(path).encode()))

    def correct(self):
        """Applies the corrector set on this context to the current state (dh_correct)."""
        self._check(self.lib.dh_correct(self.ctx))

    def correct_every_step(self, on: bool):
        """Every later step applies the corrector on the device (dh_set_correct_every_step)."""
        self._check(self.lib.dh_set_correct_every_step(self.ctx, int(on)))

    def profile(self, enable: bool):
        self._check(self.lib.dh_profile_enable(self.ctx, int(enable)))

    def profile_read(self, kind: str):
        n = C.c_longlong()
        ms = C.c_double()
        self._check(self.lib.dh_profile_read(self.ctx, _lib.KERNEL_KINDS[kind], C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._check(self.lib.dh_launch_count(self.ctx, C.byref(n)))
        return n.value
