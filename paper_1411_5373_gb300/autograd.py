"""Differentiable FDMT: a torch.autograd.Function over the C ABI.

Forward is ``fdmt_execute`` on w .* x; backward is ``fdmt_adjoint``, which
returns both the input gradient w .* FDMT^T(g) and the per-channel weight
gradient <x[k], FDMT^T(g)[k]> from the library's own kernels.
"""
from __future__ import annotations

import torch

from .plan import Plan


class FDMTFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, weights, plan: Plan):
        if plan.dtype == "u8":
            raise ValueError("the differentiable transform needs a float plan")
        x = x.contiguous()
        w = None if weights is None else weights.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(x, w)
        ctx.has_w = w is not None
        return plan.execute(x, weights=w)

    @staticmethod
    def backward(ctx, grad_out):
        x, w = ctx.saved_tensors
        plan = ctx.plan
        gw = None
        if ctx.has_w and ctx.needs_input_grad[1]:
            gw = torch.empty(plan.nf, dtype=torch.float32, device=x.device)
        gx = plan.adjoint(grad_out.contiguous().float(), x=x, weights=w, grad_weights=gw)
        return (gx if ctx.needs_input_grad[0] else None), gw, None


def fdmt(x, plan: Plan, weights=None):
    """Differentiable A = FDMT(weights .* x) for a float plan."""
    return FDMTFunction.apply(x, weights, plan)
