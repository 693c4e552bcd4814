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

Flux form (Sec. 7's learned flux, applied after the step): W3 has 15 output channels,
y[5 a + c] the flux of field c through the face i + 1/2 along axis a (x, y, z), and the
correction is dU_c(i) = -s_c sum_a (y_{a,c}(i) - y_{a,c}(i - e_a)): a periodic divergence, so
every conserved total is unchanged.

Solver-in-the-loop rollout loss (Sec. 7): from U_0, each step applies the solver step H_s and
then the correction, U_s = C(H_s(U_{s-1})) for s = 1..S, and
L = (1/S) sum_s mean over fields c and cells of ((U_s - T_s) / w_c)^2 against reference states
T_s, with per-field weights w.  Reverse mode of this function is the gradient the rollout
training follows.

Pins: tests/test_oracle_corrector.py (brute-force convolution, delta-kernel translation,
translation equivariance, gelu values and derivative, bf16 rounding of hand values, zero
network = identity map, hand-evaluated layer composition of a centre-tap network (bf16
roundings, GELU on layers 1-2 only, normalisation, output scale), hand-evaluated floors with
each one binding alone and together, flux form: exact conservation and a single face moving
mass between two cells, the transposed divergence, and the rollout gradient against finite
differences).
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


def flux_divergence(y: torch.Tensor) -> torch.Tensor:
    """-sum_a (y_{a,c}(i) - y_{a,c}(i - e_a)) for the 15-channel flux output, per field c."""
    out = torch.zeros((5,) + tuple(y.shape[1:]), dtype=y.dtype)
    for a in range(3):
        dim = 3 - a                      # x is the last tensor dimension of a (5, nz, ny, nx) field set
        ya = y[5 * a:5 * a + 5]
        out = out - (ya - torch.roll(ya, 1, dims=dim))
    return out


def correction(U: torch.Tensor, p: dict, mu, sigma, out_scale=None) -> torch.Tensor:
    """dU before the floors: s * y (state form, 5 outputs) or s * divergence(y) (flux form,
    15 outputs), s = out_scale per field (sigma when not given)."""
    s = torch.as_tensor(sigma if out_scale is None else out_scale, dtype=torch.float64).reshape(5, 1, 1, 1)
    y, _ = forward(U, p, mu, sigma)
    return s * (flux_divergence(y) if y.shape[0] == 15 else y)


def correct(U: torch.Tensor, p: dict, mu, sigma, rho_floor: float, T_floor: float, gamma: float,
            out_scale=None):
    """U + dU (either form), then the floors."""
    V = U + correction(U, p, mu, sigma, out_scale)
    rho = torch.clamp(V[0], min=rho_floor)
    kin = 0.5 * (V[1] ** 2 + V[2] ** 2 + V[3] ** 2) / rho
    Emin = kin + rho * T_floor / (gamma - 1.0)
    out = V.clone()
    out[0] = rho
    out[4] = torch.maximum(V[4], Emin)
    return out


def rollout_loss(U0: torch.Tensor, steps, targets, p: dict, mu, sigma, out_scale, weights,
                 rho_floor: float, T_floor: float, gamma: float) -> torch.Tensor:
    """The rollout loss above: steps[s] maps a state to the next (the solver step of interval s),
    targets[s] is T_{s+1}, weights w (5 values)."""
    w = torch.as_tensor(weights, dtype=torch.float64).reshape(5, 1, 1, 1)
    U = U0
    L = torch.zeros((), dtype=torch.float64)
    for H, T in zip(steps, targets):
        U = correct(H(U), p, mu, sigma, rho_floor, T_floor, gamma, out_scale)
        L = L + (((U - T) / w) ** 2).mean()
    return L / len(steps)
