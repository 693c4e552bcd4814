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


def _rows(shape):
    nz, ny, nx = shape
    return int(_lib.load().dh_conv_padded_rows(nx, ny, nz))


def _padded_empty(cpad, shape):
    """Zeroed bf16 buffer of the padded layout (guard rows must read zero)."""
    return torch.zeros(cpad // 8 * _rows(shape) * 8, dtype=torch.bfloat16, device="cuda")


def _unpad(buf, cpad, shape):
    nz, ny, nx = shape
    out = torch.empty(nx * ny * nz, cpad, dtype=torch.bfloat16, device="cuda")
    assert _lib.load().dh_conv_unpad(_ptr(buf), cpad, nx, ny, nz, _ptr(out), None) == 0
    torch.cuda.synchronize()
    return out


def _conv(act, cin_pad, packed, nout_pad, bias, mode, shape, z_in=None, n_real=32, keep=None):
    """act: padded layout.  Returns (out, z_out) with bf16 outputs unpadded to [cell][32];
    keep (a list) receives the padded output buffer."""
    lib = _lib.load()
    nz, ny, nx = shape
    ncell = nx * ny * nz
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    z_out = None
    if mode == 0:
        out = _padded_empty(32, shape)
        z_out = torch.empty(ncell, 32, dtype=torch.float32, device="cuda")
    elif mode == 1:
        out = torch.empty(n_real, ncell, dtype=torch.float32, device="cuda")
    else:
        out = _padded_empty(32, shape)
    b = bias.float().contiguous().cuda() if bias is not None else None
    st = lib.dh_conv3d_bf16(_ptr(act), cin_pad, _ptr(packed), nout_pad, _ptr(b), mode, _ptr(z_in),
                            _ptr(out), _ptr(z_out), n_real, nx, ny, nz, _ptr(err), None)
    assert st == 0, lib.dh_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0, "bounded wait gave up"
    if keep is not None:
        keep.append(out)
    if mode != 1:
        out = _unpad(out, 32, shape)
    return out, z_out


def _act(x, cpad):
    """(c, nz, ny, nx) float64 -> bf16 padded layout with cpad channels on the GPU."""
    c = x.shape[0]
    shape = tuple(x.shape[1:])
    nz, ny, nx = shape
    flat = torch.zeros(x[0].numel(), cpad, dtype=torch.float64)
    flat[:, :c] = x.reshape(c, -1).t()
    cl = flat.to(torch.bfloat16).cuda().contiguous()
    buf = _padded_empty(cpad, shape)
    assert _lib.load().dh_conv_pad(_ptr(cl), cpad, nx, ny, nz, _ptr(buf), None) == 0
    torch.cuda.synchronize()
    return buf


def _planar(a, c, shape):
    return a.float().cpu().double()[:, :c].t().reshape((c,) + shape)


SHAPES = [(8, 16, 16), (16, 8, 32), (5, 7, 9), (64, 64, 64)]   # (5, 7, 9): 315 cells, ragged tiles


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


def test_long_rows_take_one_window_stage():
    """Rows of 176 cells leave room for one shared-memory window stage only (the tile's windows
    load after the previous tile's MMAs): the hidden layer still matches the oracle."""
    shape = (4, 5, 176)
    g = torch.Generator().manual_seed(13)
    x = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(32, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    b = torch.randn(32, generator=g, dtype=torch.float64) * 0.1
    out, z = _conv(_act(x, 32), 32, _pack(W, 0), 32, b, 0, shape)
    zr = oc.conv3d_periodic(x, oc.bf16(W), b)
    zg = _planar(z, 32, shape)
    assert float((zg - zr).abs().max() / zr.abs().max()) < 1e-5


def test_padded_output_layout_images_and_guards():
    """The GELU output in the padded layout: every halo row equals the periodic image it
    stands for, and the guard rows stay zero."""
    shape = (5, 7, 9)
    nz, ny, nx = shape
    g = torch.Generator().manual_seed(11)
    x = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(32, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    keep = []
    out, _ = _conv(_act(x, 32), 32, _pack(W, 0), 32, None, 0, shape, keep=keep)
    R = _rows(shape)
    buf = keep[0].float().cpu().reshape(4, R, 8)
    PX, PY, PZ = nx + 2, ny + 2, nz + 2
    guard = (R - PX * PY * PZ) // 2
    assert torch.count_nonzero(buf[:, :guard]) == 0 and torch.count_nonzero(buf[:, guard + PX * PY * PZ:]) == 0
    vol = buf[:, guard:guard + PX * PY * PZ].reshape(4, PZ, PY, PX, 8)
    cells = out.float().cpu().reshape(nz, ny, nx, 4, 8).permute(3, 0, 1, 2, 4)
    idx = lambda n: torch.tensor([(i - 1) % n for i in range(n + 2)])
    expect = cells[:, idx(nz)][:, :, idx(ny)][:, :, :, idx(nx)]
    assert torch.equal(vol, expect)


def test_periodic_shift_equivariance_is_bitwise():
    """Each output row is computed by the same sequence of MMAs wherever its tile falls, so a
    periodic shift of the input shifts the output bit for bit."""
    shape = (8, 16, 16)
    g = torch.Generator().manual_seed(12)
    x = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(32, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    b = torch.randn(32, generator=g, dtype=torch.float64) * 0.1
    pk = _pack(W, 0)
    _, z0 = _conv(_act(x, 32), 32, pk, 32, b, 0, shape)
    shift = (3, 5, 7)
    _, z1 = _conv(_act(torch.roll(x, shift, dims=(1, 2, 3)), 32), 32, pk, 32, b, 0, shape)
    a = _planar(z0, 32, shape)
    c = _planar(z1, 32, shape)
    assert torch.equal(torch.roll(a, shift, dims=(1, 2, 3)), c)


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_output_layer_32_to_5_linear(shape):
    g = torch.Generator().manual_seed(2)
    x = oc.bf16(torch.randn((32,) + shape, generator=g, dtype=torch.float64))
    W = torch.randn(5, 32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.05
    b = torch.randn(5, generator=g, dtype=torch.float64) * 0.1
    y, _ = _conv(_act(x, 32), 32, _pack(W, 0), 16, b, 1, shape, n_real=5)
    yr = oc.conv3d_periodic(x, oc.bf16(W), b)
    yg = y.double().cpu().reshape((5,) + shape)
    assert float((yg - yr).abs().max() / yr.abs().max()) < 1e-5


@pytest.mark.parametrize("shape", SHAPES[:3])
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


def _wgrad(x, gr, cin_pad, g_stride, cout, shape):
    lib = _lib.load()
    nz, ny, nx = shape
    nctas = 148
    mt = (27 * cin_pad + 127) // 128
    nout_pad = 32 if cout > 16 else 16
    partial = torch.empty(nctas * mt * 128 * nout_pad, dtype=torch.float32, device="cuda")
    dW = torch.empty(cout * x.shape[0] * 27, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    a_dev = _act(x, cin_pad)      # keep the device buffers alive until the kernel has run
    g_dev = _act(gr, g_stride)
    st = lib.dh_conv3d_wgrad_bf16(_ptr(a_dev), cin_pad, x.shape[0], _ptr(g_dev),
                                  g_stride, cout, nx, ny, nz, _ptr(partial), nctas, _ptr(dW), _ptr(err), None)
    assert st == 0, lib.dh_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return dW.double().cpu().reshape(cout, x.shape[0], 3, 3, 3)


@pytest.mark.parametrize("cin,cout,shape", [(5, 32, (8, 16, 16)), (32, 32, (8, 16, 16)),
                                            (32, 5, (16, 8, 32)), (32, 32, (5, 7, 9)),
                                            (32, 32, (64, 64, 64))])
def test_weight_gradient(cin, cout, shape):
    g = torch.Generator().manual_seed(5)
    x = oc.bf16(torch.randn((cin,) + shape, generator=g, dtype=torch.float64))
    gr = oc.bf16(torch.randn((cout,) + shape, generator=g, dtype=torch.float64))
    got = _wgrad(x, gr, 8 if cin <= 8 else 32, 8 if cout <= 8 else 32, cout, shape)
    ref = oc.conv3d_weight_grad(x, gr, cout)
    assert float((got - ref).norm() / ref.norm()) < 1e-5


@pytest.mark.parametrize("cin,cout,nctas", [(32, 32, 148), (5, 32, 37), (32, 5, 9)])
def test_weight_gradient_reduction_order(cin, cout, nctas):
    """The per-CTA partials are added in the documented fixed order: warp w of a (channel, tap)
    block sums the CTAs b = w, w + 8, ... in increasing b in float64, and the eight sums combine
    as ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7)); the float32 result is checked bit for bit
    against that sum of the partials the kernel left in the scratch buffer."""
    lib = _lib.load()
    shape = (6, 8, 16)
    nz, ny, nx = shape
    cin_pad, g_stride = (8 if cin <= 8 else 32), (8 if cout <= 8 else 32)
    g = torch.Generator().manual_seed(11)
    x = oc.bf16(torch.randn((cin,) + shape, generator=g, dtype=torch.float64))
    gr = oc.bf16(torch.randn((cout,) + shape, generator=g, dtype=torch.float64))
    mt = (27 * cin_pad + 127) // 128
    nout_pad = 32 if cout > 16 else 16
    partial = torch.empty(nctas * mt * 128 * nout_pad, dtype=torch.float32, device="cuda")
    dW = torch.empty(cout * cin * 27, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    a_dev, g_dev = _act(x, cin_pad), _act(gr, g_stride)
    st = lib.dh_conv3d_wgrad_bf16(_ptr(a_dev), cin_pad, cin, _ptr(g_dev), g_stride, cout, nx, ny, nz,
                                  _ptr(partial), nctas, _ptr(dW), _ptr(err), None)
    assert st == 0, lib.dh_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    P = partial.cpu().numpy().astype(np.float64).reshape(nctas, mt * 128, nout_pad)
    expect = np.empty((cout, cin, 27), dtype=np.float32)
    for tap in range(27):
        for c in range(cin):
            row = P[:, tap * cin_pad + c, :cout]
            s = []
            for w in range(8):
                acc = np.zeros(cout)
                for b in range(w, nctas, 8):
                    acc = acc + row[b]
                s.append(acc)
            r = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]))
            expect[:, c, tap] = r.astype(np.float32)
    got = dW.cpu().numpy().reshape(cout, cin, 27)
    assert np.array_equal(got.view(np.uint32), expect.view(np.uint32))
    # and the sum is the weight gradient
    ref = oc.conv3d_weight_grad(x, gr, cout)
    assert float((torch.from_numpy(got).double().reshape(ref.shape) - ref).norm() / ref.norm()) < 1e-5


def _net_params(seed):
    from paper_2512_13403_b300 import corrector as cr
    p = cr.init_params(seed, out_scale=1.0)
    g = torch.Generator().manual_seed(seed)
    p = p + 0.01 * torch.randn(p.shape, generator=g)   # nonzero biases too
    return p, cr.unflatten(p.double())


def test_network_forward_and_backward_against_oracle():
    from paper_2512_13403_b300 import corrector as cr
    shape = (8, 16, 16)
    params, pd = _net_params(3)
    U = torch.from_numpy(__import__("paper_2512_13403_b300").inputs.decaying_turbulence(shape, seed=1, sigma=0.5, mach=1.0, p_sigma=0.3))
    mu = [float(U[c].mean()) for c in range(5)]
    sigma = [float(U[c].std()) for c in range(5)]
    net = cr.Network(shape)
    net.set_params(params, mu, sigma)
    Ug = U.float().cuda().contiguous()
    y = net.forward(Ug)
    yr, cache = oc.forward(U.float().double(), pd, mu, sigma)
    assert float((y.double().cpu() - yr).norm() / yr.norm()) < 1e-2
    # backward of the mean-squared error against a target, vs reverse-mode AD of the oracle with
    # the BF16 roundings passed straight through
    tgt = yr + 0.1 * torch.randn(yr.shape, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    grads = torch.zeros(cr.NPARAM, dtype=torch.float32, device="cuda")
    # residual target (U_target - U_in)/s with U_in = 0 and s = sigma gives tgt itself
    zero = torch.zeros_like(Ug)
    sg = torch.tensor(sigma, dtype=torch.float64).reshape(5, 1, 1, 1)
    loss = net.backward(zero, (tgt * sg).float().cuda().contiguous(), grads)
    q = {k: v.clone().requires_grad_(True) for k, v in pd.items()}
    st = lambda t: t + (oc.bf16(t) - t).detach()
    mu_t = torch.tensor(mu, dtype=torch.float64).reshape(5, 1, 1, 1)
    sg_t = torch.tensor(sigma, dtype=torch.float64).reshape(5, 1, 1, 1)
    x0 = oc.bf16((U.float().double() - mu_t) / sg_t)
    h1 = st(oc.gelu(oc.conv3d_periodic(x0, st(q["W1"]), q["b1"])))
    h2 = st(oc.gelu(oc.conv3d_periodic(h1, st(q["W2"]), q["b2"])))
    yy = oc.conv3d_periodic(h2, st(q["W3"]), q["b3"])
    L = ((yy - tgt) ** 2).mean()
    L.backward()
    assert loss == pytest.approx(float(L.detach()), rel=2e-2)
    gg = cr.unflatten(grads.double().cpu())
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        ref = q[k].grad
        assert float((gg[k] - ref).norm() / ref.norm()) < 3e-2, k


def test_zero_network_is_identity_and_floors():
    from paper_2512_13403_b300 import corrector as cr
    shape = (8, 16, 16)
    net = cr.Network(shape)
    net.set_params(torch.zeros(cr.NPARAM), [0.0] * 5, [1.0] * 5, [1.0] * 5)
    U = torch.from_numpy(__import__("paper_2512_13403_b300").inputs.decaying_turbulence(shape, seed=2, sigma=0.5, mach=1.0)).float().cuda().contiguous()
    V = U.clone()
    net.correct_state(V, 1e-6, 0.05, 5 / 3)
    assert torch.equal(V, U)
    # a state below the floors is lifted onto them
    W = U.clone()
    W[0, 0, 0, 0] = -1.0
    W[4, 1, 1, 1] = 0.0
    net.correct_state(W, 1e-3, 0.05, 5 / 3)
    assert float(W[0, 0, 0, 0]) == pytest.approx(1e-3)
    kin = 0.5 * float(W[1, 1, 1, 1] ** 2 + W[2, 1, 1, 1] ** 2 + W[3, 1, 1, 1] ** 2) / float(W[0, 1, 1, 1])
    assert float(W[4, 1, 1, 1]) >= kin + float(W[0, 1, 1, 1]) * 0.05 * 1.5 * (1 - 1e-6)


def test_adam_matches_definition():
    from paper_2512_13403_b300 import corrector as cr
    g = torch.Generator().manual_seed(7)
    p0 = torch.randn(1000, generator=g)
    p = p0.clone().cuda()
    opt = cr.Adam(p, lr=1e-2)
    m = torch.zeros(1000, dtype=torch.float64)
    v = torch.zeros(1000, dtype=torch.float64)
    pr = p0.double().clone()
    for t in range(1, 4):
        grad = torch.randn(1000, generator=g)
        opt.step(grad.cuda())
        gd = grad.double()
        m = 0.9 * m + 0.1 * gd
        v = 0.999 * v + 0.001 * gd * gd
        pr = pr - 1e-2 * (m / (1 - 0.9 ** t)) / (torch.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    torch.cuda.synchronize()
    assert torch.allclose(p.double().cpu(), pr, rtol=1e-5, atol=1e-6)
