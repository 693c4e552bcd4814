"""Helpers shared by the GPU parity tests (CUDA path via the C ABI vs the CPU oracle)."""
import numpy as np
import torch


def solver(shape, precision="f64", **kw):
    from paper_2512_13403_b300.solver import Config, Solver
    return Solver(Config(shape=shape, precision=precision, **kw))


def to_gpu(U, precision):
    dt = torch.float64 if precision == "f64" else torch.float32
    return torch.as_tensor(np.ascontiguousarray(U)).to(dtype=dt, device="cuda").contiguous()


def rel_linf(gpu, ref):
    """Per-field max |gpu - ref| / max |ref|."""
    g = gpu.detach().double().cpu()
    r = torch.as_tensor(ref).double()
    out = []
    for f in range(g.shape[0]):
        den = float(r[f].abs().max())
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
