"""Differentiable Poisson solve: torch.autograd.Function over the C ABI.

The solve is affine in the source, psi = A_psi f + c and op = A_op f + c'
(the constants come only from boundary data), so the backward pass needs
nothing from the forward pass: dL/df = A_psi^T g_psi + A_op^T g_op is one
transposed solve (sf_solve_adjoint) on the incoming gradients.  The padded
spectral buffers of the forward solve are therefore never stored; the adjoint
recomputes its own transforms from the gradients.
"""
from __future__ import annotations

import torch

from . import Plan


class _PoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, plan: Plan):
        ctx.plan = plan
        psi, opo = plan.empty_outputs()
        plan.execute(f.contiguous(), psi, opo)
        if opo is None:
            return psi
        return psi, opo

    @staticmethod
    def backward(ctx, *grads):
        plan = ctx.plan
        g_psi = grads[0].contiguous() if grads[0] is not None else None
        g_op = None
        if len(grads) > 1 and grads[1] is not None:
            g_op = grads[1].contiguous()
        if g_psi is None and g_op is None:
            return None, None
        g_f = plan.adjoint(g_psi, g_op)
        return g_f, None


def poisson_solve(f: torch.Tensor, plan: Plan):
    """psi (and the operator output) of lap(psi) = rhs_scale f, differentiable in f."""
    return _PoissonSolve.apply(f, plan)
