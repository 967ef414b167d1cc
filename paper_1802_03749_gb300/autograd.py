"""res_calc as a differentiable PyTorch operation.

Forward: ``loop_res_calc`` (res = sum of edge increments).  Backward:
``loop_adjoint``, the hand-written adjoint, giving the gradients with
respect to q and x; adt is treated as a fixed input (no gradient).  Both
calls take the same plan, built with both maps written (``AirfoilPlans(...,
adjoint=True)``), so forward and backward share one numbering and one
two-layer colouring.
"""
from __future__ import annotations

import torch

from . import loop_adjoint, loop_res_calc


class ResCalc(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, adt, plan, gam=1.4, eps=0.05):
        res = torch.zeros_like(q)
        loop_res_calc(plan, x.contiguous(), q.contiguous(), adt.contiguous(), res, gam, eps)
        ctx.save_for_backward(x, q, adt)
        ctx.plan = plan
        ctx.consts = (gam, eps)
        return res

    @staticmethod
    def backward(ctx, res_bar):
        x, q, adt = ctx.saved_tensors
        gam, eps = ctx.consts
        q_bar = torch.zeros_like(q)
        x_bar = torch.zeros_like(x)
        loop_adjoint(ctx.plan, x.contiguous(), q.contiguous(), adt.contiguous(), res_bar.contiguous(), q_bar,
                     x_bar, gam, eps)
        return x_bar, q_bar, None, None, None, None


def res_calc(x, q, adt, plan, gam=1.4, eps=0.05):
    """Differentiable res_calc(x, q, adt) in plan numbering and layout."""
    return ResCalc.apply(x, q, adt, plan, gam, eps)
