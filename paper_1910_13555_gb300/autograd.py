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


class BlockSparseContractFn(torch.autograd.Function):
    """R_data = execute(contraction plan) with T1, T2 (and R_in) data bound to the given
    tensors; the backward runs the plan's adjoint kernels, which give dT1 and dT2 on the
    existing block patterns of T1 and T2 (and dR_in = beta dR), each in its tensor's
    packing."""

    @staticmethod
    def forward(ctx, t1_data, t2_data, rin_data, plan, alpha, beta, precision):
        res = bst.bst_plan_result_tensor(plan.handle)
        _, _, ne = bst.bst_tensor_info(res)
        r = torch.empty(max(ne, 1), dtype=torch.float64, device=t1_data.device)
        bst.bst_tensor_bind_data(res, r)
        bst.bst_multiply_execute(plan.handle, alpha, beta, precision, 1)
        ctx.plan = plan
        ctx.alpha, ctx.beta = alpha, beta
        ctx.has_rin = rin_data is not None
        ctx.shapes = (t1_data.shape, t2_data.shape, None if rin_data is None else rin_data.shape)
        ctx.dev = t1_data.device
        return r

    @staticmethod
    def backward(ctx, gr):
        gr = gr.contiguous()
        s1, s2, sr = ctx.shapes
        d1 = torch.empty(s1, dtype=torch.float64, device=ctx.dev)
        d2 = torch.empty(s2, dtype=torch.float64, device=ctx.dev)
        dri = torch.empty(sr, dtype=torch.float64, device=ctx.dev) if ctx.has_rin else None
        bst.bst_plan_adjoint(ctx.plan.handle, gr, d1, d2, dri, ctx.alpha, ctx.beta)
        return d1, d2, dri, None, None, None, None


def contract(T1: bst.Tensor, T2: bst.Tensor, c1, c2, f1, f2, result_order=None,
             R_in: bst.Tensor | None = None, alpha=1.0, beta=0.0, eps=0.0,
             precision=bst.BST_FP64, device=0):
    """Differentiable R = alpha sum_{contracted} T1 T2 + beta R_in (paper Sec. 4).
    T1.data / T2.data (and R_in.data) may require grad.  Returns (R data tensor, plan);
    the result's block index is plan's result tensor (bst_plan_result_tensor)."""
    plan = bst.contract_plan(T1, T2, c1, c2, f1, f2, result_order, R_in, eps, device)
    r = BlockSparseContractFn.apply(T1.data, T2.data, None if R_in is None else R_in.data, plan,
                                    alpha, beta, precision)
    return r, plan

