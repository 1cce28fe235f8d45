"""torch.autograd.Function around the C ABI: the direct solve is the forward pass and
the hand-written Paraexp adjoint (pxa_solve_adjoint) is the backward pass.

Only argument marshalling happens here. The context keeps what the adjoint needs
from the forward solve (q(T) and the adjoint source, or the Burgers trajectory /
checkpoints). If the context ran another forward solve before this backward, the
direct solve is recomputed from the saved control first.
"""
from __future__ import annotations

import torch

from . import pxa as X


class ParaexpSolve(torch.autograd.Function):
    """J = ParaexpSolve.apply(control, context, mode): the objective of one direct solve
    (0-dim float64 tensor). d J / d control comes from the adjoint solve of the same mode."""

    @staticmethod
    def forward(ctx, control, context, mode):
        if not control.is_contiguous():
            control = control.contiguous()
        context.set_control(control)
        J = context.solve_direct(mode)
        context._direct_token = getattr(context, "_direct_token", 0) + 1
        ctx.context = context
        ctx.mode = mode
        ctx.token = context._direct_token
        ctx.save_for_backward(control)
        return torch.tensor(J, dtype=torch.float64, device=control.device)

    @staticmethod
    def backward(ctx, gJ):
        (control,) = ctx.saved_tensors
        context = ctx.context
        if getattr(context, "_direct_token", None) != ctx.token:
            # another forward used the context in between: recompute the direct solve
            context.set_control(control)
            context.solve_direct(ctx.mode)
            context._direct_token = getattr(context, "_direct_token", 0) + 1
            ctx.token = context._direct_token
        grad = torch.empty_like(control)
        context.solve_adjoint(ctx.mode, grad)
        return gJ * grad, None, None


def objective(control, context, mode=X.PARAEXP):
    """Differentiable objective J(control) on a configured pxa Context."""
    return ParaexpSolve.apply(control, context, mode)
