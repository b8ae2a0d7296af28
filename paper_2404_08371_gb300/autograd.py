"""Differentiable operator apply y = A(k) u for coefficient fields (torch.autograd).

Forward: y = A(k) u through the library's apply.  Backward, for an upstream
gradient g = dL/dy:
  dL/du = A(k)^T g = A(k) g          (the bilinear form is symmetric, so is A_D)
  dL/dk_m = g^T (dA/dk_m) u          (A is linear in k; the library's adjoint
                                       kernel evaluates it element by element,
                                       recomputing the element data)
Nothing of the forward pass is stored besides u and k.

Vectors are packed library vectors.  On meshes with several macros a point
shared by macros is stored once per macro; the gradients returned are the
gradients of the distinct-point functions, written into every copy, which is
exact when the loss reads every distinct point once.
"""
from __future__ import annotations

import torch

from . import Operator


class _ApplyAk(torch.autograd.Function):
    @staticmethod
    def forward(ctx, op: Operator, u: torch.Tensor, k: torch.Tensor):
        u = u.contiguous()
        k = k.contiguous()
        op.set_field(k)
        y = op.apply(u)
        ctx.op = op
        ctx.save_for_backward(u, k)
        return y

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        u, k = ctx.saved_tensors
        op = ctx.op
        op.set_field(k)
        g = g.contiguous()
        du = op.apply(g) if ctx.needs_input_grad[1] else None
        dk = op.adjoint_coeff(u, g) if ctx.needs_input_grad[2] else None
        return None, du, dk


def apply_ak(op: Operator, u: torch.Tensor, k: torch.Tensor) -> torch.Tensor:
    """y = A(k) u, differentiable in u and k; op must have a field coefficient of k's space."""
    if op.field is None:
        raise ValueError("apply_ak needs an operator with a coefficient field")
    return _ApplyAk.apply(op, u, k)
