"""Helpers shared by the GPU parity tests (CUDA path via the C ABI vs the CPU oracle)."""
import numpy as np
import torch


def solver(shape, precision="f64", **kw):
    from paper_2512_13403_b300.solver import Config, Solver
    return Solver(Config(shape=shape, precision=precision, **kw))


def to_gpu(U, precision):
    dt = torch.float64 if precision == "f64" else torch.float32
    return torch.as_tensor(np.ascontiguousarray(U)).to(dtype=dt, device="cuda").contiguous()


def rel_linf(gpu, ref, own_scale=False):
    """Per-field max |gpu - ref| / scale.  The scale of a field is max |ref_f|; with
    own_scale=False (default) the three momentum components of a 5-field state share the scale
    max |m| of the momentum vector, so a component that is identically zero in the reference
    (round-off noise on the GPU) is measured against the momentum it belongs to."""
    g = gpu.detach().double().cpu()
    r = torch.as_tensor(ref).double()
    vec = g.shape[0] == 5 and not own_scale
    mag = float(torch.sqrt(r[1] ** 2 + r[2] ** 2 + r[3] ** 2).max()) if vec else 0.0
    out = []
    for f in range(g.shape[0]):
        den = mag if (vec and f in (1, 2, 3)) else float(r[f].abs().max())
        num = float((g[f] - r[f]).abs().max())
        out.append(num / den if den > 0 else num)
    return out


def rel_l1(gpu, ref):
    """Per-field sum |gpu - ref| / sum |ref|."""
    g = gpu.detach().double().cpu()
    r = torch.as_tensor(ref).double()
    out = []
    for f in range(g.shape[0]):
        den = float(r[f].abs().sum())
        num = float((g[f] - r[f]).abs().sum())
        out.append(num / den if den > 0 else num)
    return out


def rel_l1_vector_scaled(gpu, ref):
    """Per-field sum |gpu - ref| / scale, where the scale of rho and E is their own L1 norm and
    the scale of each momentum component is the L1 norm of the momentum magnitude |m| (the
    three components of one vector share one physical scale)."""
    g = gpu.detach().double().cpu()
    r = torch.as_tensor(ref).double()
    mag = float(torch.sqrt(r[1] ** 2 + r[2] ** 2 + r[3] ** 2).sum())
    out = []
    for f in range(5):
        den = mag if f in (1, 2, 3) else float(r[f].abs().sum())
        out.append(float((g[f] - r[f]).abs().sum()) / den)
    return out
