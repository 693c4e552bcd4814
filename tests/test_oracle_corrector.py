"""Pins of the oracle's corrector network (CPU only)."""
import math

import numpy as np
import pytest
import torch

from oracle import corrector as oc


def _brute_conv(x, W):
    cin, nz, ny, nx = x.shape
    cout = W.shape[0]
    out = torch.zeros(cout, nz, ny, nx, dtype=torch.float64)
    for o in range(cout):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    s = 0.0
                    for c in range(cin):
                        for a in range(3):
                            for b in range(3):
                                for d in range(3):
                                    s += float(W[o, c, a, b, d]) * float(
                                        x[c, (k + a - 1) % nz, (j + b - 1) % ny, (i + d - 1) % nx])
                    out[o, k, j, i] = s
    return out


def test_periodic_conv_matches_brute_force():
    g = torch.Generator().manual_seed(0)
    x = torch.randn(2, 3, 4, 5, generator=g, dtype=torch.float64)
    W = torch.randn(3, 2, 3, 3, 3, generator=g, dtype=torch.float64)
    assert torch.allclose(oc.conv3d_periodic(x, W), _brute_conv(x, W), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("off", [(-1, 0, 1), (1, 1, 1), (0, -1, 0)])
def test_delta_kernel_translates(off):
    g = torch.Generator().manual_seed(1)
    x = torch.randn(3, 5, 6, 7, generator=g, dtype=torch.float64)
    W = torch.zeros(3, 3, 3, 3, 3, dtype=torch.float64)
    dz, dy, dx = off
    for c in range(3):
        W[c, c, dz + 1, dy + 1, dx + 1] = 1.0
    y = oc.conv3d_periodic(x, W)
    assert torch.equal(y, torch.roll(x, shifts=(-dz, -dy, -dx), dims=(1, 2, 3)))


def test_translation_equivariance():
    g = torch.Generator().manual_seed(2)
    x = torch.randn(2, 6, 6, 6, generator=g, dtype=torch.float64)
    W = torch.randn(4, 2, 3, 3, 3, generator=g, dtype=torch.float64)
    a = oc.conv3d_periodic(torch.roll(x, (2, -1, 3), (1, 2, 3)), W)
    b = torch.roll(oc.conv3d_periodic(x, W), (2, -1, 3), (1, 2, 3))
    assert torch.allclose(a, b, rtol=1e-13, atol=1e-13)


def test_gelu_values_and_derivative():
    z = torch.tensor([0.0, 1.0, -1.0, 2.5], dtype=torch.float64)
    # gelu(z) = z Phi(z); Phi(1) = 0.8413447460685429 (standard normal CDF)
    exp = [0.0, 0.8413447460685429, -1.0 + 0.8413447460685429, 2.5 * 0.9937903346742238]
    assert oc.gelu(z).tolist() == pytest.approx(exp, abs=1e-15)
    h = 1e-6
    fd = (oc.gelu(z + h) - oc.gelu(z - h)) / (2 * h)
    assert torch.allclose(oc.gelu_grad(z), fd, atol=1e-9)


def test_bf16_rounding_hand_values():
    x = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7 + 2.0 ** -8, 3.0e38],
                     dtype=torch.float64)
    # 8 significand bits: halfway cases go to even
    assert oc.bf16(x).tolist()[:3] == [1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -6]


def test_zero_network_is_identity():
    g = torch.Generator().manual_seed(3)
    shape = (4, 4, 4)
    U = torch.rand((5,) + shape, generator=g, dtype=torch.float64) + 1.0
    U[4] = U[4] + 5.0  # well above the floor
    p = {"W1": torch.zeros(32, 5, 3, 3, 3, dtype=torch.float64), "b1": torch.zeros(32, dtype=torch.float64),
         "W2": torch.zeros(32, 32, 3, 3, 3, dtype=torch.float64), "b2": torch.zeros(32, dtype=torch.float64),
         "W3": torch.zeros(5, 32, 3, 3, 3, dtype=torch.float64), "b3": torch.zeros(5, dtype=torch.float64)}
    out = oc.correct(U, p, [0.0] * 5, [1.0] * 5, 1e-6, 0.05, 5 / 3)
    assert torch.equal(out, U)


def test_data_and_weight_gradients_by_duality():
    g = torch.Generator().manual_seed(4)
    x = torch.randn(3, 4, 5, 4, generator=g, dtype=torch.float64)
    W = torch.randn(2, 3, 3, 3, 3, generator=g, dtype=torch.float64)
    dy = torch.randn(2, 4, 5, 4, generator=g, dtype=torch.float64)
    lhs = float((dy * oc.conv3d_periodic(x, W)).sum())
    assert lhs == pytest.approx(float((oc.conv3d_data_grad(dy, W) * x).sum()), rel=1e-12)
    assert lhs == pytest.approx(float((oc.conv3d_weight_grad(x, dy, 2) * W).sum()), rel=1e-12)
