"""Small fixed workloads for profiling one kernel family under a profiler (ncu), each a few
seconds and a few hundred MB on the device.

    python -m paper_2512_13403_b300.profile_cases adjoint [n]     # dh_adjoint_advance, 2 steps
    python -m paper_2512_13403_b300.profile_cases corrector [n]   # 3 network forwards + 1 backward
    python -m paper_2512_13403_b300.profile_cases stage [n]       # 3 forward steps, driven cooling box
    python -m paper_2512_13403_b300.profile_cases selfgrav [n]    # 4 steps, gravity + forcing + cooling
"""
from __future__ import annotations

import sys
import time

import torch

from . import inputs
from .solver import Config, Solver


def adjoint(n: int = 128):
    s = Solver(Config(shape=(n, n, n), precision="f32"))
    s.init_state(torch.from_numpy(inputs.decaying_turbulence((n, n, n), seed=2, sigma=0.5, mach=2.0))
                 .float().cuda().contiguous())
    lam = torch.randn((5, n, n, n), generator=torch.Generator().manual_seed(0)).cuda()
    out = s.adjoint_advance(2, 2, lam)
    torch.cuda.synchronize()
    print("adjoint", n, float(out.abs().sum()))


def corrector(n: int = 64):
    from . import corrector as cr
    U = torch.from_numpy(inputs.decaying_turbulence((n, n, n), seed=1, sigma=0.5, mach=1.0, p_sigma=0.3)) \
        .float().cuda().contiguous()
    mu = [float(U[c].mean()) for c in range(5)]
    sg = [float(U[c].std()) for c in range(5)]
    net = cr.Network((n, n, n))
    net.set_params(cr.init_params(0, out_scale=1.0).cuda(), mu, sg)
    grads = torch.zeros(cr.NPARAM, device="cuda")
    for _ in range(3):
        net.forward(U)
    net.backward(U, U, grads)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.forward(U)
    torch.cuda.synchronize()
    print("corrector", n, "forward+sync ms", (time.perf_counter() - t0) * 1e3)


def stage(n: int = 128):
    s = Solver(Config(shape=(n, n, n), precision="f32", forcing=True, cooling=True, t_floor=0.05))
    s.init_state(torch.from_numpy(inputs.cooling_box((n, n, n))).float().cuda().contiguous())
    s.advance(3)
    torch.cuda.synchronize()
    print("stage", n, s.time())


def selfgrav(n: int = 1024):
    from . import inputs as _in
    cfg = Config(shape=(n, n, n), precision="f32", forcing=True, cooling=True, t_floor=0.05,
                 gravity=True, four_pi_G=1.0, mg_tol=1e-6, mg_max_cycles=30)
    s = Solver(cfg)
    U0 = _in.self_gravitating_box_device((n, n, n), seed=5, sigma=1.0)
    s.init_state(U0)
    del U0
    torch.cuda.empty_cache()
    s.advance(4)
    torch.cuda.synchronize()
    print("selfgrav", n, s.time(), s.mg_stats())


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "stage"
    size = int(sys.argv[2]) if len(sys.argv) > 2 else None
    fn = {"adjoint": adjoint, "corrector": corrector, "stage": stage, "selfgrav": selfgrav}[case]
    fn() if size is None else fn(size)
