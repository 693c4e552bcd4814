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


def _params(form, seed=0, scale=0.3):
    g = torch.Generator().manual_seed(seed)
    k = 15 if form == "flux" else 5
    shapes = {"W1": (32, 5, 3, 3, 3), "b1": (32,), "W2": (32, 32, 3, 3, 3), "b2": (32,),
              "W3": (k, 32, 3, 3, 3), "b3": (k,)}
    return {n: scale * torch.randn(s, generator=g, dtype=torch.float64) / math.sqrt(27 * (s[1] if len(s) > 1 else 1))
            for n, s in shapes.items()}


def test_flux_divergence_conserves_every_total():
    g = torch.Generator().manual_seed(3)
    y = torch.randn(15, 5, 6, 7, generator=g, dtype=torch.float64)
    d = oc.flux_divergence(y)
    assert d.shape == (5, 5, 6, 7)
    for c in range(5):
        assert abs(float(d[c].sum())) < 1e-12 * float(y.abs().sum())


@pytest.mark.parametrize("a,c", [(0, 0), (1, 3), (2, 4)])
def test_single_face_flux_moves_mass_between_two_cells(a, c):
    """Flux f through the face i + 1/2 along axis a: cell i loses f, cell i + e_a gains f."""
    y = torch.zeros(15, 4, 5, 6, dtype=torch.float64)
    k, j, i = 3, 4, 5                     # a cell on the upper boundary of every axis
    y[5 * a + c, k, j, i] = 2.5
    d = oc.flux_divergence(y)
    nxt = [k, j, i]
    nxt[2 - a] = (nxt[2 - a] + 1) % (4, 5, 6)[2 - a]
    expect = torch.zeros_like(d)
    expect[c, k, j, i] = -2.5
    expect[c, nxt[0], nxt[1], nxt[2]] = 2.5
    assert torch.equal(d, expect)


def test_transposed_flux_divergence_is_forward_difference():
    """(d D / d y)^T g at (a, c, i) = g_c(i + e_a) - g_c(i): the rule the GPU output gradient
    follows."""
    gen = torch.Generator().manual_seed(5)
    y = torch.randn(15, 4, 5, 6, generator=gen, dtype=torch.float64, requires_grad=True)
    gg = torch.randn(5, 4, 5, 6, generator=gen, dtype=torch.float64)
    (gy,) = torch.autograd.grad((oc.flux_divergence(y) * gg).sum(), y)
    for a in range(3):
        dim = 3 - a
        expect = torch.roll(gg, -1, dims=dim) - gg
        assert torch.allclose(gy[5 * a:5 * a + 5], expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("form", ["state", "flux"])
def test_rollout_gradient_matches_finite_differences(form, monkeypatch):
    """Reverse mode of the rollout loss (two solver steps, each followed by the correction)
    against central differences along a random parameter direction, BF16 rounding off."""
    from oracle import hydro
    from paper_2512_13403_b300 import inputs
    monkeypatch.setattr(oc, "bf16", lambda t: t)
    shape = (6, 6, 6)
    U0 = torch.from_numpy(inputs.decaying_turbulence(shape, seed=4, sigma=0.3, mach=0.5, p_sigma=0.2))
    dx = (1 / 6, 1 / 6, 1 / 6)
    steps = [lambda U: hydro.rk2_step(U, 2e-3, 5 / 3, dx)] * 2
    T = [U0 + 0.01 * torch.randn(U0.shape, generator=torch.Generator().manual_seed(s), dtype=torch.float64)
         for s in (1, 2)]
    mu = [float(U0[c].mean()) for c in range(5)]
    sg = [float(U0[c].std()) + 0.1 for c in range(5)]
    out = [0.01] * 5
    w = [0.1, 0.2, 0.2, 0.2, 0.3]
    p = _params(form, seed=1)
    q = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    L = oc.rollout_loss(U0, steps, T, q, mu, sg, out, w, 1e-9, 1e-6, 5 / 3)
    L.backward()
    gen = torch.Generator().manual_seed(7)
    dirn = {k: torch.randn(v.shape, generator=gen, dtype=torch.float64) for k, v in p.items()}
    ad = sum(float((q[k].grad * dirn[k]).sum()) for k in p)
    eps = 1e-5
    f = lambda t: float(oc.rollout_loss(U0, steps, T, {k: p[k] + t * dirn[k] for k in p}, mu, sg, out,
                                        w, 1e-9, 1e-6, 5 / 3))
    fd = (f(eps) - f(-eps)) / (2 * eps)
    assert ad == pytest.approx(fd, rel=1e-6)


def _centre_tap(M):
    """3x3x3 kernels whose only nonzero tap is the centre one: the convolution is then the
    per-cell linear map M."""
    M = torch.tensor(M, dtype=torch.float64)
    W = torch.zeros(M.shape + (3, 3, 3), dtype=torch.float64)
    W[..., 1, 1, 1] = M
    return W


def _t(v):
    return torch.tensor(v, dtype=torch.float64)


def test_layer_composition_hand_values():
    """A 5 -> 1 -> 1 -> 5 network with centre-tap kernels (a pointwise MLP), evaluated by hand
    through normalise -> bf16 -> conv -> GELU -> bf16 -> conv -> GELU -> bf16 -> conv -> * s
    (Sec. 7 corrector; the GELU values are the standard normal CDF tabulated at 1 and -1).

    Cell A, U = (3, 1, 0, 0, 5), mu = (1, 0, 0, 0, 1), sigma = (2, 1, 1, 1, 4):
      x0 = ((3-1)/2, 1, 0, 0, (5-1)/4) = (1, 1, 0, 0, 1)          (exact in bf16)
      z1 = 1 * x0[0] + 0 = 1;  gelu(1) = Phi(1) = 0.8413447460685429
      h1 = bf16(0.84134...) = 215/256 = 0.83984375   (215.38 ulps of 2^-8, rounded down)
      z2 = 1 * h1 + 41/256 = 1;  h2 = 215/256 again
      y  = (h2 + 0.5, 0, 0, 0, -2 h2) = (1.33984375, 0, 0, 0, -1.6796875)   (no GELU here)
      U' = U + s y, s = (0.5, 1, 1, 1, 0.25): rho' = 3.669921875, E' = 4.580078125
      (kinetic energy 0.5/3.67 is far below E', so the floors do not act).
    Cell B, U = (-1, 1, 0, 0, 5): x0[0] = -1, z1 = -1, gelu(-1) = Phi(1) - 1 = -0.15865525393145707
      h1 = bf16(.) = -162/1024 = -0.158203125   (162.46 ulps of 2^-10, rounded down)
      z2 = -162/1024 + 164/1024 = 2^-9;  gelu(2^-9) = 2^-9 Phi(2^-9) = 2^-10 (1 + 1.6e-3)
      h2 = bf16(.) = 2^-10   (below half an ulp, 2^-18, above 2^-10)
      y  = (2^-10 + 0.5, 0, 0, 0, -2^-9) = (0.5009765625, 0, 0, 0, -0.001953125)
      rho = -1 + 0.5 * 0.5009765625 < rho_floor = 1e-3  ->  rho' = 1e-3
      E' = max(5 - 2^-9 / 4, 0.5 * 1^2 / 1e-3 + 1e-3 * 0.05 / (2/3)) = 500.000075.
    A GELU after the last layer, a missing bf16 rounding, (U/sigma - mu) for the normalisation
    or a missing output scale each changes one of these numbers."""
    p = {"W1": _centre_tap([[1.0, 0, 0, 0, 0]]), "b1": _t([0.0]),
         "W2": _centre_tap([[1.0]]), "b2": _t([41 / 256]),
         "W3": _centre_tap([[1.0], [0], [0], [0], [-2.0]]), "b3": _t([0.5, 0, 0, 0, 0])}
    U = torch.zeros(5, 1, 1, 2, dtype=torch.float64)
    U[:, 0, 0, 0] = _t([3.0, 1.0, 0.0, 0.0, 5.0])
    U[:, 0, 0, 1] = _t([-1.0, 1.0, 0.0, 0.0, 5.0])
    mu, sg, s = [1.0, 0, 0, 0, 1.0], [2.0, 1, 1, 1, 4.0], [0.5, 1, 1, 1, 0.25]
    y, t = oc.forward(U, p, mu, sg)
    assert t["h1"][0, 0, 0].tolist() == [0.83984375, -0.158203125]
    assert t["h2"][0, 0, 0].tolist() == [0.83984375, 2.0 ** -10]
    assert y[:, 0, 0, 0].tolist() == [1.33984375, 0.0, 0.0, 0.0, -1.6796875]
    assert y[:, 0, 0, 1].tolist() == [0.5009765625, 0.0, 0.0, 0.0, -0.001953125]
    out = oc.correct(U, p, mu, sg, 1e-3, 0.05, 5 / 3, out_scale=s)
    assert out[:, 0, 0, 0].tolist() == [3.669921875, 1.0, 0.0, 0.0, 4.580078125]
    assert out[:, 0, 0, 1].tolist()[:4] == [1e-3, 1.0, 0.0, 0.0]
    assert float(out[4, 0, 0, 1]) == pytest.approx(500.000075, rel=1e-15)


def test_floors_hand_values():
    """The floors after the correction (Sec. 7 with the temperature floor of Sec. 4.3): rho is
    raised to rho_floor first, then E to |m|^2 / (2 rho') + rho' T_floor / (gamma - 1) with the
    floored rho'.  All weights zero, so y = b3 and U' = U + b3 (s = 1).  rho_floor = 0.01,
    T_floor = 0.05, gamma = 5/3, so the thermal floor is 0.075 rho'.  b3 = (-1, 0.1, 0, 0, -0.5).
      A: U = (0.5, 0.2, -0.1, 0, 0.6) -> (-0.5, 0.3, -0.1, 0, 0.1); rho' = 0.01;
         E' = 0.5 (0.09 + 0.01) / 0.01 + 0.01 * 0.075 = 5.00075        (both floors bind)
      B: U = (2, 0.2, 0.2, 0.1, 0.6) -> (1, 0.3, 0.2, 0.1, 0.1);
         E' = 0.5 (0.09 + 0.04 + 0.01) / 1 + 0.075 = 0.145             (only the energy floor)
      C: U = (3, 0, 0, 0, 2) -> (2, 0.1, 0, 0, 1.5);
         floor energy 0.005 / 2 + 0.15 = 0.1525 < 1.5, so E' = 1.5     (neither)
    Kinetic energy taken from the unfloored rho, or E floored before rho, gives a negative
    floor energy in A and leaves E' = 0.1 there."""
    z = lambda *s: torch.zeros(s, dtype=torch.float64)
    p = {"W1": z(32, 5, 3, 3, 3), "b1": z(32), "W2": z(32, 32, 3, 3, 3), "b2": z(32),
         "W3": z(5, 32, 3, 3, 3), "b3": _t([-1.0, 0.1, 0.0, 0.0, -0.5])}
    U = torch.zeros(5, 1, 1, 3, dtype=torch.float64)
    U[:, 0, 0, 0] = _t([0.5, 0.2, -0.1, 0.0, 0.6])
    U[:, 0, 0, 1] = _t([2.0, 0.2, 0.2, 0.1, 0.6])
    U[:, 0, 0, 2] = _t([3.0, 0.0, 0.0, 0.0, 2.0])
    out = oc.correct(U, p, [0.0] * 5, [1.0] * 5, 0.01, 0.05, 5 / 3, out_scale=[1.0] * 5)
    expect = [[0.01, 0.3, -0.1, 0.0, 5.00075],
              [1.0, 0.3, 0.2, 0.1, 0.145],
              [2.0, 0.1, 0.0, 0.0, 1.5]]
    for i, e in enumerate(expect):
        assert out[:, 0, 0, i].tolist() == pytest.approx(e, rel=1e-14, abs=1e-15)
