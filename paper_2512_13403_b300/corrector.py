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

FORMS = {"state": 0, "flux": 1}
NOUT = {"state": 5, "flux": 15}


def layout(form: str = "state"):
    k = NOUT[form]
    return [("W1", (32, 5, 3, 3, 3)), ("b1", (32,)), ("W2", (32, 32, 3, 3, 3)), ("b2", (32,)),
            ("W3", (k, 32, 3, 3, 3)), ("b3", (k,))]


def nparam(form: str = "state") -> int:
    return int(sum(np.prod(s) for _, s in layout(form)))


NPARAM = nparam("state")
LAYOUT = layout("state")


def init_params(seed: int = 0, out_scale: float = 0.1, form: str = "state") -> torch.Tensor:
    """Seeded fan-in uniform initialisation (float32, CPU); the output layer is scaled down so the
    untrained correction starts small."""
    g = np.random.default_rng(seed)
    parts = []
    for name, shape in layout(form):
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
    assert flat.size == nparam(form)
    return torch.from_numpy(flat)


def unflatten(p: torch.Tensor) -> dict:
    form = "flux" if p.numel() == nparam("flux") else "state"
    out, o = {}, 0
    for name, shape in layout(form):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


class Network:
    """One dh_cnn for a grid of shape (nz, ny, nx) on the current CUDA stream."""

    def __init__(self, shape, stream=None, form: str = "state"):
        self.lib = _lib.load()
        self.form = form
        self.nparam = nparam(form)
        assert self.lib.dh_cnn_param_count_form(FORMS[form]) == self.nparam
        self.shape = tuple(shape)
        nz, ny, nx = self.shape
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(self.lib.dh_cnn_create_form(nx, ny, nz, FORMS[form], C.c_void_p(self.stream.cuda_stream),
                                          C.byref(h)))
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
        """The network outputs y (5 or 15 planes); keeps the activations for backward / vjp."""
        assert U.dtype == torch.float32 and U.is_cuda and U.is_contiguous()
        y = torch.empty((NOUT[self.form],) + self.shape, dtype=torch.float32, device=U.device)
        check(self.lib.dh_cnn_forward(self.h, C.c_void_p(U.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def vjp(self, dL_dcorr: torch.Tensor, grads: torch.Tensor, want_input: bool = True):
        """For the last forward: parameter gradients into grads and (optionally) returns dL/dU
        of the correction dU(U) for the upstream gradient dL_dcorr (5 planes, device)."""
        assert dL_dcorr.dtype == torch.float32 and dL_dcorr.is_cuda and dL_dcorr.is_contiguous()
        gU = torch.empty_like(dL_dcorr) if want_input else None
        check(self.lib.dh_cnn_vjp(self.h, C.c_void_p(dL_dcorr.data_ptr()), C.c_void_p(grads.data_ptr()),
                                  C.c_void_p(gU.data_ptr() if gU is not None else 0)))
        return gU

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

    def rollout_misfit(self, U: torch.Tensor, T: torch.Tensor, weights, coef: float, lam=None,
                       accumulate: bool = False, loss_acc=None):
        """dh_cnn_rollout_misfit: adds coef * sum((U - T)/w)^2 to loss_acc (a device float64
        tensor) and writes or adds its gradient into lam."""
        w = (C.c_float * 5)(*[float(v) for v in weights])
        check(self.lib.dh_cnn_rollout_misfit(
            self.h, C.c_void_p(U.data_ptr()), C.c_void_p(T.data_ptr()), w, float(coef),
            C.c_void_p(lam.data_ptr() if lam is not None else 0), int(accumulate),
            C.c_void_p(loss_acc.data_ptr() if loss_acc is not None else 0)))

    def floor_vjp(self, V: torch.Tensor, lam: torch.Tensor, rho_floor: float, T_floor: float,
                  gamma: float):
        """dh_cnn_floor_vjp: lam (dL/dU' after the floors) becomes dL/d(V + dU), for the last
        forward, which must have been on V."""
        check(self.lib.dh_cnn_floor_vjp(self.h, C.c_void_p(V.data_ptr()), C.c_void_p(lam.data_ptr()),
                                        float(rho_floor), float(T_floor), float(gamma)))

    def field_moments(self, A: torch.Tensor, B: torch.Tensor = None):
        """dh_cnn_field_moments over the samples of A (or A - B): (means, standard deviations),
        five each."""
        assert A.dtype == torch.float32 and A.is_cuda and A.is_contiguous()
        count = A.numel() // (5 * int(np.prod(self.shape)))
        out = (C.c_double * 10)()
        check(self.lib.dh_cnn_field_moments(self.h, C.c_void_p(A.data_ptr()),
                                            C.c_void_p(B.data_ptr() if B is not None else 0),
                                            count, out))
        return list(out[:5]), list(out[5:])


def axpy(a: float, x: torch.Tensor, y: torch.Tensor):
    """y += a x on the current stream (dh_axpy)."""
    assert x.numel() == y.numel() and x.dtype == y.dtype == torch.float32
    check(_lib.load().dh_axpy(x.numel(), float(a), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream)))


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
