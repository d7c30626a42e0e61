"""torch.autograd.Function around the volumetric PROPELLER operator.

forward(V) = prop_forward (y = A V); backward(g_y) = prop_adjoint (A^H g_y).
With torch's convention for complex tensors (the gradient of a real loss is
dL/dRe + i dL/dIm), the vector-Jacobian product of the linear map A is
A^H g_y.  Nothing is saved for backward but the plan: the adjoint of a
linear operator needs no forward state, and the oversampled grid is
recomputed inside the adjoint rather than stored.
"""
from __future__ import annotations

import torch

from .binding import Plan


class PropOp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.forward(V.contiguous())

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        return ctx.plan.adjoint(gy.contiguous()), None


def prop_apply(V: torch.Tensor, plan: Plan) -> torch.Tensor:
    """y = A V with autograd support (complex64 CUDA tensors)."""
    return PropOp.apply(V, plan)
