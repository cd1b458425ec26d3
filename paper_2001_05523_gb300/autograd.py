"""torch.autograd wrapper of the H^2 product.

H2Apply.apply(x, op) returns y = A x through h2bem_apply; its backward maps the
incoming gradient g to A^T g through h2bem_apply_transpose (the transposed H^2
pass: V and W exchanged, transposed block lists and nearfield), so that
d<w, A x>/dx = A^T w.  Both directions run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import h2bem as H


class H2Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, op: "H.Operator") -> torch.Tensor:
        if x.dtype != torch.float64 or not x.is_cuda:
            raise ValueError("x must be a float64 CUDA tensor of shape (nrhs, n)")
        xc = x.contiguous()
        y = torch.empty_like(xc)
        H.h2bem_apply(op.op, xc, y)
        ctx.op = op
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        g = gy.contiguous()
        gx = torch.empty_like(g)
        H.h2bem_apply_transpose(ctx.op.op, g, gx)
        return gx, None


class H2ApplyShape(torch.autograd.Function):
    """y = G(X) x, differentiable in x and in the vertex coordinates X (single
    layer; the operator's cluster tree and block lists stay fixed).  The
    backward pass returns G^T g for x and, for X, the shape gradient
    d<g, G(X) x>/dX from h2bem_grad."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, vertices: torch.Tensor, op) -> torch.Tensor:
        xc = x.contiguous()
        y = torch.empty_like(xc)
        H.h2bem_apply(op.op, xc, y)
        ctx.op = op
        ctx.save_for_backward(xc, vertices)
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        xc, vertices = ctx.saved_tensors
        g = gy.contiguous()
        gx = torch.empty_like(g)
        gX = torch.empty((vertices.shape[0], 3), dtype=torch.float64, device=g.device)
        H.h2bem_grad(ctx.op.op, g, xc, gX, gx)
        return gx, gX.to(vertices.dtype), None


def h2_apply_shape(x: torch.Tensor, vertices: torch.Tensor, op) -> torch.Tensor:
    """Differentiable y = G(X) x in x and X; `op` must have been built from the
    values of `vertices` (shape (nv, 3))."""
    if x.dim() == 1:
        return H2ApplyShape.apply(x[None, :], vertices, op)[0]
    return H2ApplyShape.apply(x, vertices, op)


def h2_apply(x: torch.Tensor, op: "H.Operator") -> torch.Tensor:
    """Differentiable y = A x; x of shape (nrhs, n) or (n,)."""
    if x.dim() == 1:
        return H2Apply.apply(x[None, :], op)[0]
    return H2Apply.apply(x, op)
