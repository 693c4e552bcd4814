"""Oracle: residual 3D convolutional corrector (Sec. 7 closure idea with the 3D CNN of the
benchmark set-up).  Test infrastructure only.

Network (channel counts 5 -> 32 -> 32 -> 5, 3x3x3 kernels, periodic padding as in Sec. 7.1):
  x0 = bf16((U - mu) / sigma)
  z1 = conv(x0, bf16(W1)) + b1,  h1 = bf16(gelu(z1))
  z2 = conv(h1, bf16(W2)) + b2,  h2 = bf16(gelu(z2))
  y  = conv(h2, bf16(W3)) + b3
  U' = U + s * y (s a per-channel output scale, by default sigma), then rho >= rho_floor and
       E raised where needed so that
       E - |m|^2 / (2 rho) >= rho T_floor / (gamma - 1).
BF16 rounding is round-to-nearest-even of the float64 value; products and sums are float64
(the tensor cores accumulate in float32, so the two agree to float32 rounding before each
BF16 rounding).  gelu is the exact erf form.  conv is cross-correlation,
out[o, z, y, x] = sum_{i, a, b, c} W[o, i, a, b, c] in[i, z + a - 1, y + b - 1, x + c - 1].

Pins: tests/test_oracle_corrector.py (brute-force convolution, delta-kernel translation,
translation equivariance, gelu values and derivative, bf16 rounding of hand values, zero
network = identity map).
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F


def bf16(x: torch.Tensor) -> torch.Tensor:
    return x.to(torch.bfloat16).to(torch.float64)


def conv3d_periodic(x: torch.Tensor, W: torch.Tensor, b=None) -> torch.Tensor:
    """x: (cin, nz, ny, nx), W: (cout, cin, 3, 3, 3) -> (cout, nz, ny, nx), periodic."""
    xp = F.pad(x[None], (1, 1, 1, 1, 1, 1), mode="circular")
    return F.conv3d(xp, W, bias=b)[0]


def conv3d_data_grad(dy: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """Gradient of sum(dy * conv3d_periodic(x, W)) with respect to x."""
    x = torch.zeros((W.shape[1],) + tuple(dy.shape[1:]), dtype=dy.dtype, requires_grad=True)
    (g,) = torch.autograd.grad(conv3d_periodic(x, W), x, grad_outputs=dy)
    return g


def conv3d_weight_grad(x: torch.Tensor, dy: torch.Tensor, cout: int) -> torch.Tensor:
    """Gradient of sum(dy * conv3d_periodic(x, W)) with respect to W."""
    W = torch.zeros((cout, x.shape[0], 3, 3, 3), dtype=x.dtype, requires_grad=True)
    (g,) = torch.autograd.grad(conv3d_periodic(x, W), W, grad_outputs=dy)
    return g


def gelu(z: torch.Tensor) -> torch.Tensor:
    return 0.5 * z * (1.0 + torch.erf(z / math.sqrt(2.0)))


def gelu_grad(z: torch.Tensor) -> torch.Tensor:
    return 0.5 * (1.0 + torch.erf(z / math.sqrt(2.0))) + z * torch.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(U: torch.Tensor, p: dict, mu, sigma):
    """Returns y (5, ...) and the intermediate tensors."""
    mu = torch.as_tensor(mu, dtype=torch.float64).reshape(5, 1, 1, 1)
    sigma = torch.as_tensor(sigma, dtype=torch.float64).reshape(5, 1, 1, 1)
    x0 = bf16((U - mu) / sigma)
    z1 = conv3d_periodic(x0, bf16(p["W1"]), p["b1"])
    h1 = bf16(gelu(z1))
    z2 = conv3d_periodic(h1, bf16(p["W2"]), p["b2"])
    h2 = bf16(gelu(z2))
    y = conv3d_periodic(h2, bf16(p["W3"]), p["b3"])
    return y, dict(x0=x0, z1=z1, h1=h1, z2=z2, h2=h2)


def correct(U: torch.Tensor, p: dict, mu, sigma, rho_floor: float, T_floor: float, gamma: float,
            out_scale=None):
    """U + s * y with s = out_scale (per channel; sigma when not given), then the floors."""
    s = torch.as_tensor(sigma if out_scale is None else out_scale, dtype=torch.float64).reshape(5, 1, 1, 1)
    y, _ = forward(U, p, mu, sigma)
    V = U + s * y
    rho = torch.clamp(V[0], min=rho_floor)
    kin = 0.5 * (V[1] ** 2 + V[2] ** 2 + V[3] ** 2) / rho
    Emin = kin + rho * T_floor / (gamma - 1.0)
    out = V.clone()
    out[0] = rho
    out[4] = torch.maximum(V[4], Emin)
    return out
