"""Batched products in one persistent launch (bst_batch_*), its CUDA-graph capture, and
the emulated-FP64 scaling modes, against the CPU oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import batched

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _problems(n=6):
    return batched(nprob=n, nmin=100, nmax=600, occ_min=0.01, occ_max=0.08)


def _setup(probs):
    mats, plans = [], []
    for p in probs:
        A, B = to_lib(p.A), to_lib(p.B)
        plan = bst.multiply_plan(A, B, None, p.eps)
        plan.alloc_result()
        mats.append((A, B))
        plans.append(plan)
    return mats, plans


def _results(plans):
    out = []
    for pl in plans:
        n = pl.result.info[3]
        out.append(pl.result.data[:n].cpu().numpy().copy())
    return out


@pytest.mark.parametrize("prec", [bst.BST_FP64, bst.BST_FP64_EMU_BF16])
def test_batch_matches_single_and_oracle(prec):
    import torch
    probs = _problems()
    mats, plans = _setup(probs)
    alphas = np.linspace(0.5, 1.5, len(plans))
    betas = np.zeros(len(plans))
    batch = bst.bst_batch_create(bst.context(), [p.handle for p in plans])
    bst.bst_batch_execute(batch, alphas, betas, prec)
    torch.cuda.synchronize()
    got = _results(plans)
    for q, pl in enumerate(plans):
        pl.execute(alphas[q], 0.0, prec, 1)
    torch.cuda.synchronize()
    single = _results(plans)
    tol = 1e-12 if prec == bst.BST_FP64 else 1e-11
    for q, p in enumerate(probs):
        assert (got[q] == single[q]).all()  # same kernels, same summation order
        ref = oracle.multiply(p.A, p.B, None, alphas[q], 0.0, p.eps)
        assert rel_fro(got[q], ref["data"]) <= tol
    bst.bst_batch_destroy(batch)


@pytest.mark.parametrize("prec", [bst.BST_FP64, bst.BST_FP64_EMU_BF16])
def test_batch_graph_capture_and_replay(prec):
    import torch
    probs = _problems(4)
    mats, plans = _setup(probs)
    alphas, betas = np.ones(len(plans)), np.zeros(len(plans))
    batch = bst.bst_batch_create(bst.context(), [p.handle for p in plans])
    bst.bst_batch_execute(batch, alphas, betas, prec)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cs):
        bst.bst_batch_execute(batch, alphas, betas, prec, stream=cs)
    for pl in plans:
        pl.result.data.fill_(np.nan)
    g.replay()
    torch.cuda.synchronize()
    tol = 1e-12 if prec == bst.BST_FP64 else 1e-11
    got = _results(plans)
    for q, p in enumerate(probs):
        ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
        assert rel_fro(got[q], ref["data"]) <= tol
    # new operand values in place (sign flips keep every block norm, so the plans'
    # filter decisions stay valid), replay again: the graph reads the current data
    for (A, B), p in zip(mats, probs):
        A.data.mul_(-1.0)
        p.A.data *= -1.0
    g.replay()
    torch.cuda.synchronize()
    got = _results(plans)
    for q, p in enumerate(probs):
        ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
        assert rel_fro(got[q], ref["data"]) <= tol
    bst.bst_batch_destroy(batch)


@pytest.mark.parametrize("mode", [0, 1])
def test_emulated_scaling_modes(mode):
    from gpu_util import run_multiply
    from paper_1910_13555_gb300.workloads import banded
    ctx = bst.context()
    old = bst.bst_tune_get(ctx, bst.BST_TUNE_EMU_ROW_SCALE)
    try:
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_ROW_SCALE, mode)
        for p in (banded(seed=3, nb=300, decay=40.0, value_decay=8.0, eps=1e-8),
                  _problems(2)[1]):
            ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
            got = run_multiply(p, precision=bst.BST_FP64_EMU_BF16, stacks=False)
            assert rel_fro(got["data"], ref["data"]) <= 1e-11
    finally:
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_ROW_SCALE, old)
