"""torch.autograd.Function around dh_advance / dh_adjoint_advance.

Forward: U_n = H^n(U_0) through the CUDA library.  Backward: the hand adjoint with
checkpoint-every-k recomputation (dh_adjoint_advance), which replays the forward from U_0 and
returns dL/dU_0 for the incoming dL/dU_n; the time steps are held at the forward's values (the
stopped dt gradient of App. A.4).  Only marshalling happens here.
"""
from __future__ import annotations

import torch


class AdvanceFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0: torch.Tensor, solver, n_steps: int, ckpt_every: int):
        solver.init_state(U0.detach().contiguous())
        solver.advance(n_steps)
        ctx.solver = solver
        ctx.n_steps = n_steps
        ctx.ckpt_every = ckpt_every
        ctx.save_for_backward(U0.detach().clone())
        return solver.get_state()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (U0,) = ctx.saved_tensors
        s = ctx.solver
        s.init_state(U0)
        g = s.adjoint_advance(ctx.n_steps, ctx.ckpt_every, grad_out.contiguous())
        return g, None, None, None


def advance(U0: torch.Tensor, solver, n_steps: int, ckpt_every: int = 10) -> torch.Tensor:
    """Differentiable n-step update of U0 (shape (5, nz, ny, nx), solver precision, on CUDA)."""
    return AdvanceFunction.apply(U0, solver, n_steps, ckpt_every)
