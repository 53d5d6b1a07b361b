"""The rectangular case S_B << S_A, S_C (paper Sec. 3.2: a small B between a tall A and
a tall C) and a rank-4 x rank-3 contraction over two index pairs with a permuted matrix
view and a reordered result (paper Sec. 4), on the GPU against the CPU oracle: small
instances in full (patterns bit-exact, values within 1e-12 / 1e-11), the full-size
workloads on sampled output blocks that the oracle computes exactly."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, run_multiply, to_lib
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import rank4, rect_case2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _gather(data, offs, lens):
    import torch
    idx = np.concatenate([np.arange(o, o + n) for o, n in zip(offs, lens)])
    return data[torch.as_tensor(idx, device=data.device)].cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(bst.BST_FP64, 1e-12), (bst.BST_FP64_EMU_BF16, 1e-11)])
def test_rect_case2_small(prec, tol):
    p = rect_case2(seed=21, nm=600, nk=40, window=10, p=0.3, bwin=6, bp=0.5)
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    got = run_multiply(p, precision=prec, stacks=prec == bst.BST_FP64)
    assert (got["rows"] == ref["rows"]).all() and (got["cols"] == ref["cols"]).all()
    assert rel_fro(got["data"], ref["data"]) <= tol
    if prec == bst.BST_FP64:
        for key in ("a_off", "b_off", "c_off"):
            assert (got[key] == ref[key]).all()


def test_rect_case2_full_size_sampled():
    import torch
    p = rect_case2()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps)
    C = plan.alloc_result()
    rows, cols, offs = C.index()
    rng = np.random.default_rng(3)
    sel = np.sort(rng.choice(len(rows), 64, replace=False))
    ref, present = oracle.multiply_sample(p.A, p.B, None, 1.0, 0.0, p.eps, rows[sel], cols[sel],
                                          row_sizes=p.A.row_sizes, col_sizes=p.B.col_sizes)
    assert present.all()
    lens = p.A.row_sizes[rows[sel]].astype(np.int64) * p.B.col_sizes[cols[sel]]
    for prec, tol in ((bst.BST_FP64, 1e-12), (bst.BST_FP64_EMU_BF16, 1e-11)):
        plan.execute(1.0, 0.0, prec, 1)
        torch.cuda.synchronize()
        assert rel_fro(_gather(C.data, offs[sel], lens), ref) <= tol
    # stack count = sum over inner blocks of nnz(A column) * nnz(B row)
    ca = np.bincount(p.A.cols, minlength=len(p.A.col_sizes)).astype(np.int64)
    rb = np.bincount(p.B.rows, minlength=len(p.B.row_sizes)).astype(np.int64)
    assert plan.stats()["n_stack"] == int((ca * rb).sum())


def _contract(w, prec=bst.BST_FP64):
    import torch
    t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data)
    t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data)
    plan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, precision=prec)
    torch.cuda.synchronize()
    return plan, (t1, t2)


@pytest.mark.parametrize("prec,tol", [(bst.BST_FP64, 1e-12), (bst.BST_FP64_EMU_BF16, 1e-11)])
def test_rank4_small(prec, tol):
    w = rank4(seed=22, nP=24, nao=20, window=5, p4=0.3, p3=0.4)
    ref = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    plan, _ = _contract(w, prec)
    idx, off = plan.result.index()
    ne = plan.result.info[2]
    assert (idx == ref["index"]).all() and (off == ref["offsets"]).all()
    assert rel_fro(plan.result.data[:ne].cpu().numpy(), ref["data"]) <= tol


def test_rank4_full_size_sampled_and_adjoint():
    import torch
    w = rank4()
    plan, (t1, t2) = _contract(w)
    R = plan.result
    idx, offs = R.index()
    rs = [w.T1.block_sizes[1], w.T2.block_sizes[2], w.T1.block_sizes[3]]  # (mu, sig, lam)
    rng = np.random.default_rng(4)
    sel = np.sort(rng.choice(len(idx), 32, replace=False))
    ref, present = oracle.contract_sample(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order,
                                          None, 1.0, 0.0, 0.0, idx[sel], rs)
    assert present.all()
    lens = np.ones(len(sel), np.int64)
    for d in range(3):
        lens *= rs[d][idx[sel, d]].astype(np.int64)
    assert rel_fro(_gather(R.data, offs[sel], lens), ref) <= 1e-12
    # adjoint of L = 1/2 ||R||^2: <dV, V> = <dU, U> = ||R||^2 (bilinearity)
    ne = R.info[2]
    dR = R.data[:ne].clone()
    dV = torch.empty_like(t1.data)
    dU = torch.empty_like(t2.data)
    bst.bst_plan_adjoint(plan.handle, dR, dV, dU, None, 1.0, 0.0)
    torch.cuda.synchronize()
    rr = float((dR * dR).sum())
    assert abs(float((dV * t1.data).sum()) - rr) <= 1e-12 * rr
    assert abs(float((dU * t2.data).sum()) - rr) <= 1e-12 * rr
