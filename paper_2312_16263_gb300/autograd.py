"""torch.autograd.Function over the library's forward and hand-written adjoint.

    p = fwh_apply(surface, fields)       # [O][nt] float64
    loss = (p * p).sum(); loss.backward()  # fields.grad via fwh_backward

The backward calls the adjoint kernels (a gather over observers, then the
transposed spline/FD stages and the integrand Jacobian); nothing from the
forward pass is stored besides the fields themselves.
"""
from __future__ import annotations

import torch

from .api import FWH


class FWHFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fields: torch.Tensor, surface: FWH):
        fields = fields.contiguous()
        ctx.surface = surface
        ctx.save_for_backward(fields)
        return surface.forward(fields)

    @staticmethod
    def backward(ctx, grad_p: torch.Tensor):
        (fields,) = ctx.saved_tensors
        g = ctx.surface.backward(fields, grad_p.contiguous())
        return g, None


def fwh_apply(surface: FWH, fields: torch.Tensor) -> torch.Tensor:
    return FWHFunction.apply(fields, surface)
