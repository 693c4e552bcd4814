"""Python face of the corrector network in libdh.so (dh_cnn_*, dh_adam_step): marshalling only.

The network and its training step run in the library's tensor-core kernels; this module holds
device buffers (torch tensors) and passes pointers.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from ._lib import check

NPARAM = 36357
LAYOUT = [("W1", (32, 5, 3, 3, 3)), ("b1", (32,)), ("W2", (32, 32, 3, 3, 3)), ("b2", (32,)),
          ("W3", (5, 32, 3, 3, 3)), ("b3", (5,))]


def init_params(seed: int = 0, out_scale: float = 0.1) -> torch.Tensor:
    """Seeded fan-in uniform initialisation (float32, CPU); the output layer is scaled down so the
    untrained correction starts small."""
    g = np.random.default_rng(seed)
    parts = []
    for name, shape in LAYOUT:
        if name.startswith("W"):
            fan_in = shape[1] * 27
            bound = 1.0 / math.sqrt(fan_in)
            w = g.uniform(-bound, bound, size=shape)
            if name == "W3":
                w = w * out_scale
            parts.append(w.reshape(-1))
        else:
            parts.append(np.zeros(shape))
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == NPARAM
    return torch.from_numpy(flat)


def unflatten(p: torch.Tensor) -> dict:
    out, o = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


class Network:
    """One dh_cnn for a grid of shape (nz, ny, nx) on the current CUDA stream."""

    def __init__(self, shape, stream=None):
        self.lib = _lib.load()
        assert self.lib.dh_cnn_param_count() == NPARAM
        self.shape = tuple(shape)
        nz, ny, nx = self.shape
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(self.lib.dh_cnn_create(nx, ny, nz, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.dh_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: torch.Tensor, mu, sigma, out_scale=None):
        """mu, sigma: input normalisation; out_scale: per-channel scale of the correction
        (defaults to sigma)."""
        p = params.detach().float().cuda().contiguous()
        out_scale = list(sigma) if out_scale is None else list(out_scale)
        norm = (C.c_float * 15)(*[float(x) for x in list(mu) + list(sigma) + out_scale])
        check(self.lib.dh_cnn_set_params(self.h, C.c_void_p(p.data_ptr()), norm))

    def forward(self, U: torch.Tensor) -> torch.Tensor:
        assert U.dtype == torch.float32 and U.is_cuda and U.is_contiguous()
        y = torch.empty_like(U)
        check(self.lib.dh_cnn_forward(self.h, C.c_void_p(U.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def backward(self, U_in: torch.Tensor, U_target: torch.Tensor, grads: torch.Tensor) -> float:
        """Gradient of mean((y - (U_target - U_in)/s)^2) for the last forward (on U_in)."""
        loss = C.c_double()
        check(self.lib.dh_cnn_backward(self.h, C.c_void_p(U_in.data_ptr()),
                                       C.c_void_p(U_target.data_ptr()),
                                       C.c_void_p(grads.data_ptr()), C.byref(loss)))
        return loss.value

    def correct_state(self, U: torch.Tensor, rho_floor: float, T_floor: float, gamma: float):
        check(self.lib.dh_cnn_correct_state(self.h, C.c_void_p(U.data_ptr()), float(rho_floor),
                                            float(T_floor), float(gamma)))


class Adam:
    """Moment buffers for dh_adam_step."""

    def __init__(self, params: torch.Tensor, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.p = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.t = 0
        self.lib = _lib.load()

    def step(self, grads: torch.Tensor):
        self.t += 1
        check(self.lib.dh_adam_step(C.c_void_p(self.p.data_ptr()), C.c_void_p(grads.data_ptr()),
                                    C.c_void_p(self.m.data_ptr()), C.c_void_p(self.v.data_ptr()),
                                    self.p.numel(), self.lr, self.b1, self.b2, self.eps, self.t,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream)))
