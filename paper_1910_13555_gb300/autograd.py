"""torch.autograd.Function wrappers: the forward runs the library's multiply (or
contraction) kernels, the backward its adjoint kernels (bst_plan_adjoint) -- a
sampled block-sparse product restricted to the existing block patterns of the inputs.

Gradients flow to the torch tensors that hold the inputs' packed block data."""
from __future__ import annotations

import torch

from . import bst


class BlockSparseMultiplyFn(torch.autograd.Function):
    """C_data = execute(plan) with A, B (and C_in) data bound to the given tensors."""

    @staticmethod
    def forward(ctx, a_data, b_data, cin_data, plan, alpha, beta, precision):
        res = bst.bst_plan_result(plan.handle)
        _, _, _, ne = bst.bst_matrix_info(res)
        c = torch.empty(max(ne, 1), dtype=torch.float64, device=a_data.device)
        bst.bst_matrix_bind_data(res, c)
        bst.bst_multiply_execute(plan.handle, alpha, beta, precision, 1)
        ctx.plan = plan
        ctx.alpha, ctx.beta = alpha, beta
        ctx.has_cin = cin_data is not None
        ctx.shapes = (a_data.shape, b_data.shape, None if cin_data is None else cin_data.shape)
        ctx.dev = a_data.device
        return c

    @staticmethod
    def backward(ctx, gc):
        gc = gc.contiguous()
        sa, sb, sc = ctx.shapes
        da = torch.empty(sa, dtype=torch.float64, device=ctx.dev)
        db = torch.empty(sb, dtype=torch.float64, device=ctx.dev)
        dci = torch.empty(sc, dtype=torch.float64, device=ctx.dev) if ctx.has_cin else None
        bst.bst_plan_adjoint(ctx.plan.handle, gc, da, db, dci, ctx.alpha, ctx.beta)
        return da, db, dci, None, None, None, None


def multiply(A: bst.Matrix, B: bst.Matrix, C_in: bst.Matrix | None = None, alpha=1.0, beta=0.0,
             eps=0.0, transa="N", transb="N", precision=bst.BST_FP64, device=0):
    """Differentiable C_out = alpha op(A) op(B) + beta C_in.  A.data / B.data (and
    C_in.data) may require grad.  Returns (C_out data tensor, plan)."""
    plan = bst.multiply_plan(A, B, C_in, eps, transa, transb, device)
    c = BlockSparseMultiplyFn.apply(A.data, B.data, None if C_in is None else C_in.data, plan,
                                    alpha, beta, precision)
    return c, plan
