"""PyTorch autograd wrapper: forward = fio_apply, backward = fio_apply_adjoint.

For a complex-linear operator y = L f, PyTorch's vector-Jacobian product is
L^H applied to the incoming gradient, and L^H is exactly what the library's
adjoint computes for the fast operator (Sec. 3.5).  A real f goes through the
real-input forward (fio_apply_real); its gradient is the real part of L^H
applied to the incoming gradient, as PyTorch's real-to-complex rule gives.
"""
from __future__ import annotations

import torch


class FIOApply(torch.autograd.Function):
    """out = L f with the gradient L* grad_out (both through the CUDA library)."""

    @staticmethod
    def forward(ctx, f, plan):
        ctx.plan = plan
        ctx.real = not f.is_complex()
        return plan.apply(f.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.plan.adjoint(grad_out.contiguous())
        return (g.real.contiguous() if ctx.real else g), None


class FIOAdjoint(torch.autograd.Function):
    """out = L* g with the gradient L grad_out."""

    @staticmethod
    def forward(ctx, g, plan):
        ctx.plan = plan
        return plan.adjoint(g.contiguous())

    @staticmethod
    def backward(ctx, grad_out):
        return ctx.plan.apply(grad_out.contiguous()), None


def fio_apply(f, plan):
    return FIOApply.apply(f, plan)


def fio_adjoint(g, plan):
    return FIOAdjoint.apply(g, plan)
