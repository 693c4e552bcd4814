"""tcgen05 implicit-GEMM convolutions of the corrector against the oracle's float64 convolutions
on the same BF16 operands (C ABI: dh_pack_conv_weights, dh_conv3d_bf16)."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import corrector as oc
from paper_2512_13403_b300 import _lib

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _pack(W, transpose_flip):
    lib = _lib.load()
    cout, cin = W.shape[:2]
    n_real = cin if transpose_flip else cout
    c_real = cout if transpose_flip else cin
    n_pad = 32 if n_real == 32 else 16
    k_pad = 864 if c_real > 8 else 224
    packed = torch.empty(n_pad * k_pad, dtype=torch.bfloat16, device="cuda")
    Wd = W.float().contiguous().cuda()
    assert lib.dh_pack_conv_weights(_ptr(Wd), cout, cin, transpose_flip, _ptr(packed), None) == 0
    return packed


def _conv(act, cin_pad, packed, nout_pad, bias, mode, shape, z_in=None, n_real=32):
    lib = _lib.load()
    nz, ny, nx = shape
    ncell = nx * ny * nz
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    z_out = None
    if mode == 0:
        out = torch.empty(ncell, 32, dtype=torch.bfloat16, device="cuda")
        z_out = torch.empty(ncell, 32, dtype=torch.float32, device="cuda")
    elif mode == 1:
        out = torch.empty(n_real, ncell, dtype=torch.float32, device="cuda")
    else:
        out = torch.empty(ncell, 32, dtype=torch.bfloat16, device="cuda")
    b = bias.float().contiguous().cuda() if bias is not None else None
    st = lib.dh_conv3d_bf16(_ptr(act), cin_pad, _ptr(packed), nout_pad, _ptr(b), mode, _ptr(z_in),
                            _ptr(out), _ptr(z_out), n_real, nx, ny, nz, _ptr(err), None)
    assert st == 0, lib.dh_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0, "bounded wait gave up"
    return out, z_out


def _act(x, cpad):
    """(c, nz, ny, nx) float64 -> bf16 channel-last [cell][cpad] on the GPU."""
    c = x.shape[0]
    flat = torch.zeros(x[0].numel(), cpad, dtype=torch.float64)
    flat[:, :c] = x.reshape(c, -1).t()
    return flat.to(torch.bfloat16).cuda().contiguous()


def _planar(a, c, shape):
    return a.float().cpu().double()[:, :c].t().reshape((c,) + shape)


SHAPES = [(8, 16, 16), (16, 8, 32), (64, 64, 64)]


@pytest.mark.parametrize("shape", SHAPES)
def test_first_layer_5_to_32_gelu(shape):
    g = torch.Generator().manual_seed(0)
    x = oc.bf16(torch.randn((5,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(32, 5, 3, 3, 3, generator=g, dtype=torch.float64) * 0.2
    b = torch.randn(32, generator=g, dtype=torch.float64) * 0.1
    out, z = _conv(_act(x, 8), 8, _pack(W, 0), 32, b, 0, shape)
    zr = oc.conv3d_periodic(x, oc.bf16(W), b)
    zg = _planar(z, 32, shape)
    assert float((zg - zr).abs().max() / zr.abs().max()) < 1e-5
    hg = _planar(out, 32, shape)
    hr = oc.bf16(oc.gelu(zg))  # same rounding decision in the kernel's precision
    assert float((hg - hr).abs().max()) <= 2.0 ** -7 * float(hr.abs().max())


@pytest.mark.parametrize("shape", SHAPES)
def test_hidden_layer_32_to_32_gelu(shape):
    g = torch.Generator().manual_seed(1)
    x = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(32, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    b = torch.randn(32, generator=g, dtype=torch.float64) * 0.1
    out, z = _conv(_act(x, 32), 32, _pack(W, 0), 32, b, 0, shape)
    zr = oc.conv3d_periodic(x, oc.bf16(W), b)
    zg = _planar(z, 32, shape)
    assert float((zg - zr).abs().max() / zr.abs().max()) < 1e-5


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_output_layer_32_to_5_linear(shape):
    g = torch.Generator().manual_seed(2)
    x = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(5, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    b = torch.randn(5, generator=g, dtype=torch.float64) * 0.1
    y, _ = _conv(_act(x, 32), 32, _pack(W, 0), 16, b, 1, shape, n_real=5)
    yr = oc.conv3d_periodic(x, oc.bf16(W), b)
    yg = y.double().cpu().reshape((5,) + shape)
    assert float((yg - yr).abs().max() / yr.abs().max()) < 1e-5


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_data_gradient_through_gelu(shape):
    """dz_prev = conv^T(dz, W) * gelu'(z_prev), the backward step between hidden layers."""
    g = torch.Generator().manual_seed(3)
    dz = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(32, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    zp = torch.randn((32,) + shape, generator=g, dtype=torch.float64)
    zp32 = zp.float().double()
    z_in = zp32.reshape(32, -1).t().contiguous().float().cuda()
    out, _ = _conv(_act(dz, 32), 32, _pack(W, 1), 32, None, 2, shape, z_in=z_in)
    ref = oc.conv3d_data_grad(dz, oc.bf16(W)) * oc.gelu_grad(zp32)
    got = _planar(out, 32, shape)
    assert float((got - ref).abs().max() / ref.abs().max()) < 1e-2
    assert float((got - ref).norm() / ref.norm()) < 4e-3


def test_data_gradient_of_output_layer():
    """5-channel output gradient back to the 32 hidden channels (cin_pad 8 input)."""
    shape = (8, 16, 16)
    g = torch.Generator().manual_seed(4)
    dy = oc.bf16(torch.randn((5,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(5, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    zp = torch.randn((32,) + shape, generator=g, dtype=torch.float64).float().double()
    z_in = zp.reshape(32, -1).t().contiguous().float().cuda()
    out, _ = _conv(_act(dy, 8), 8, _pack(W, 1), 32, None, 2, shape, z_in=z_in)
    ref = oc.conv3d_data_grad(dy, oc.bf16(W)) * oc.gelu_grad(zp)
    got = _planar(out, 32, shape)
    assert float((got - ref).norm() / ref.norm()) < 4e-3
