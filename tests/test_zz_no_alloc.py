"""bst_multiply_execute_static: the split-K execute for callers that may not allocate
device memory while they run (its workspace is a fixed static device array).

Checked through the C ABI against bst_multiply_execute on the same plan, on two calls
in a row (the array keeps the previous call's contents, which must not leak into the
next result), against the CPU oracle with beta != 0 and C_in and on a rank-3
contraction plan, plus the size limit (a refused call queues no work).  This file sorts last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import BSMatrix, Problem, rank3, tall_skinny

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_scratch_matches_allocating_execute_twice():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is visible")
    p = tall_skinny(seed=11, nk=4000, nmn=40, window=8, p=0.4)
    mk = lambda m: bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)
    A, B = mk(p.A), mk(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    n = C.info[3]
    split = 4
    assert split * n <= bst.bst_static_scratch_doubles()
    bst.bst_multiply_execute(plan.handle, 1.0, 0.0, bst.BST_FP64, split)
    torch.cuda.synchronize()
    ref = C.data[:n].cpu().numpy().copy()
    for call in range(2):
        C.data.fill_(np.nan)
        bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, split)
        torch.cuda.synchronize()
        got = C.data[:n].cpu().numpy()
        assert np.isfinite(got).all(), call
        assert _rel(got, ref) <= TOL_FP64, call
    # a different split on the same plan, then the original again: stale partial sums
    # from the larger call must not reach the smaller one
    bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, 8)
    bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, 2)
    torch.cuda.synchronize()
    assert _rel(C.data[:n].cpu().numpy(), ref) <= TOL_FP64


def test_static_scratch_rejects_oversize():
    import torch
    p = tall_skinny(seed=12, nk=2000, nmn=200, window=20, p=0.4)
    mk = lambda m: bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)
    A, B = mk(p.A), mk(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    n = C.info[3]
    cap = bst.bst_static_scratch_doubles()
    too_many = cap // n + 1
    if too_many > 64:
        pytest.skip("C too small to exceed the static scratch with split_k <= 64")
    with pytest.raises(bst.BstError) as e:
        bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, int(too_many))
    assert e.value.name == "BST_ERR_UNSUPPORTED"
    torch.cuda.synchronize()


def _mk(m):
    return bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)


def test_static_scratch_with_cin_against_oracle():
    """beta != 0 with C_in: the path that reads C_in, checked against the CPU oracle."""
    import torch
    p = tall_skinny(seed=13, nk=3000, nmn=40, window=8, p=0.4)
    rng = np.random.default_rng(13)
    # C_in: a random half of the blocks of the result pattern plus a few others
    full = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb)
    rs, cs = p.A.col_sizes, p.B.col_sizes
    keep = rng.random(len(full["rows"])) < 0.5
    extra_r = rng.integers(0, len(rs), 20).astype(np.int32)
    extra_c = rng.integers(0, len(cs), 20).astype(np.int32)
    pairs = sorted(set(zip(full["rows"][keep].tolist(), full["cols"][keep].tolist())) |
                   set(zip(extra_r.tolist(), extra_c.tolist())))
    ci_r = np.array([a for a, _ in pairs], np.int32)
    ci_c = np.array([b for _, b in pairs], np.int32)
    ci_d = rng.uniform(-1, 1, int((rs[ci_r].astype(np.int64) * cs[ci_c]).sum()))
    Ci = BSMatrix(rs, cs, ci_r, ci_c, ci_d)
    q = Problem(p.A, p.B, Ci, 0.75, -1.5, p.eps, p.transa, p.transb)
    ref = oracle.multiply(q.A, q.B, q.C_in, q.alpha, q.beta, q.eps, q.transa, q.transb)
    A, B, C_in = _mk(q.A), _mk(q.B), _mk(Ci)
    plan = bst.multiply_plan(A, B, C_in, q.eps, q.transa, q.transb)
    C = plan.alloc_result()
    n = C.info[3]
    assert n == len(ref["data"])
    for call in range(2):
        C.data.fill_(np.nan)
        bst.bst_multiply_execute_static(plan.handle, q.alpha, q.beta, 3)
        torch.cuda.synchronize()
        assert _rel(C.data[:n].cpu().numpy(), ref["data"]) <= TOL_FP64, call


def test_static_scratch_contraction_against_oracle():
    """A rank-3 contraction plan (its views are prepared and its result permuted by the
    call) at split_k = 3, twice, against the CPU oracle."""
    import torch
    w = rank3(nP=60, nao=80, window=10)
    t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data)
    t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data)
    plan = bst.contract_plan(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    R = plan.alloc_result()
    ref = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    n = R.info[2]
    assert n == len(ref["data"])
    for call in range(2):
        R.data.fill_(np.nan)
        bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, 3)
        torch.cuda.synchronize()
        assert _rel(R.data[:n].cpu().numpy(), ref["data"]) <= TOL_FP64, call


def test_static_refused_call_queues_nothing():
    """A call refused for its size returns before any work: C is left as it was and the
    calling thread's current device is unchanged."""
    import torch
    p = tall_skinny(seed=12, nk=2000, nmn=200, window=20, p=0.4)
    A, B = _mk(p.A), _mk(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    n = C.info[3]
    too_many = bst.bst_static_scratch_doubles() // n + 1
    if too_many > 64:
        pytest.skip("C too small to exceed the static scratch with split_k <= 64")
    C.data.fill_(7.0)
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    with pytest.raises(bst.BstError):
        bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, int(too_many))
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == dev
    assert bool((C.data[:n] == 7.0).all())
