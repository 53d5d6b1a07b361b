"""bst_multiply_execute_static: the split-K execute for callers that may not allocate
device memory while they run (its workspace is a fixed static device array).

Checked through the C ABI against bst_multiply_execute on the same plan, on two calls
in a row (the array keeps the previous call's contents, which must not leak into the
next result), plus the size limit.  This file sorts last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import tall_skinny

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
