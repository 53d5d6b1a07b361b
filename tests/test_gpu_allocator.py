"""Caller-owned device memory and host-detected failures through the C ABI.

A context created with allocator callbacks takes every device allocation of the library
from them: here they are backed by torch's caching allocator.  An allocator that fails
on its k-th call must turn into BST_ERR_ALLOC with every buffer of the failed call
handed back and the context still usable; a product whose result exceeds 2^31-1
elements is BST_ERR_OVERFLOW before any numeric work.  Also: batch executes queued back
to back with different alpha each use their own alpha."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import banded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


class TorchAllocator:
    """bst_alloc_fn / bst_free_fn backed by torch's caching allocator, allocating on the
    stream the library names.  Optionally returns NULL on its fail_at-th call."""

    def __init__(self, device=0, fail_at=None):
        self.device = device
        self.live = {}
        self.calls = 0
        self.fail_at = fail_at

    def alloc(self, nbytes, user, stream):
        import torch
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        s = (torch.cuda.ExternalStream(stream, device=self.device) if stream
             else torch.cuda.default_stream(self.device))
        with torch.cuda.stream(s):
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{self.device}")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, user, stream):
        self.live.pop(ptr)


def _mats(ctx, p):
    import torch
    out = []
    for m in (p.A, p.B):
        d = torch.as_tensor(m.data).cuda()
        out.append((bst.bst_matrix_create(ctx, m.row_sizes, m.col_sizes, m.rows, m.cols, d), d))
    return out


def _run(ctx, p):
    import torch
    (A, _), (B, _) = mats = _mats(ctx, p)
    plan = bst.bst_multiply_plan(ctx, "N", "N", A, B, None, p.eps)
    C = bst.bst_plan_result(plan)
    ne = bst.bst_matrix_info(C)[3]
    c = torch.empty(max(ne, 1), dtype=torch.float64, device="cuda")
    bst.bst_matrix_bind_data(C, c)
    bst.bst_multiply_execute(plan, 1.0, 0.0, bst.BST_FP64, 1)
    torch.cuda.synchronize()
    return plan, mats, c[:ne].cpu().numpy()


def _destroy(plan, mats):
    import torch
    torch.cuda.synchronize()
    bst.bst_plan_destroy(plan)
    for h, _ in mats:
        bst.bst_matrix_destroy(h)


def test_caller_allocator_runs_a_whole_multiply():
    p = banded(seed=21, nb=300, eps=1e-8)
    al = TorchAllocator()
    ctx = bst.bst_context_create(0, al.alloc, al.free)
    plan, mats, got = _run(ctx, p)
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    assert rel_fro(got, ref["data"]) <= 1e-12
    assert al.calls > 0 and len(al.live) > 0
    _destroy(plan, mats)
    assert al.live == {}  # the plan and the matrices returned everything
    bst.bst_context_destroy(ctx)


def test_allocator_failure_is_alloc_error_without_leak():
    p = banded(seed=22, nb=200, eps=1e-8)
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    # count the plan's allocations on a clean run
    al = TorchAllocator()
    ctx = bst.bst_context_create(0, al.alloc, al.free)
    mats = _mats(ctx, p)
    before = al.calls
    plan = bst.bst_multiply_plan(ctx, "N", "N", mats[0][0], mats[1][0], None, p.eps)
    n_plan = al.calls - before
    _destroy(plan, mats)
    bst.bst_context_destroy(ctx)
    assert n_plan >= 3
    for k in sorted({1, 2, n_plan // 2, n_plan}):
        al = TorchAllocator()
        ctx = bst.bst_context_create(0, al.alloc, al.free)
        mats = _mats(ctx, p)
        live0 = set(al.live)
        al.fail_at = al.calls + k
        with pytest.raises(bst.BstError) as e:
            bst.bst_multiply_plan(ctx, "N", "N", mats[0][0], mats[1][0], None, p.eps)
        assert e.value.name == "BST_ERR_ALLOC", (k, e.value)
        assert set(al.live) == live0, k  # the failed plan handed back what it took
        al.fail_at = None
        plan, mats2, got = _run(ctx, p)  # the context is still usable
        assert rel_fro(got, ref["data"]) <= 1e-12
        _destroy(plan, mats + mats2)
        assert al.live == {}
        bst.bst_context_destroy(ctx)


def test_overflow_is_reported_before_numeric_work():
    import torch
    ctx = bst.context()
    # a matrix of more than 2^31-1 elements: refused at creation (host check, no data)
    with pytest.raises(bst.BstError) as e:
        bst.bst_matrix_create(ctx, [50000], [50000], [0], [0])
    assert e.value.name == "BST_ERR_OVERFLOW"
    # operands that fit, a product that does not: one 50000 x 1 block times one 1 x 50000
    a = torch.ones(50000, dtype=torch.float64, device="cuda")
    b = torch.ones(50000, dtype=torch.float64, device="cuda")
    A = bst.bst_matrix_create(ctx, [50000], [1], [0], [0], a)
    B = bst.bst_matrix_create(ctx, [1], [50000], [0], [0], b)
    with pytest.raises(bst.BstError) as e:
        bst.bst_multiply_plan(ctx, "N", "N", A, B, None, 0.0)
    assert e.value.name == "BST_ERR_OVERFLOW"
    torch.cuda.synchronize()
    bst.bst_matrix_destroy(A)
    bst.bst_matrix_destroy(B)


@pytest.mark.parametrize("prec", [bst.BST_FP64, bst.BST_FP64_EMU_BF16])
def test_batch_executes_back_to_back_keep_their_alpha(prec):
    """Two batch executes queued without a synchronisation between them, the stream held
    busy so that the first parameter copy has not run when the second call rewrites the
    staging buffer: each must run with its own alpha."""
    import torch
    from paper_1910_13555_gb300.workloads import batched
    probs = batched(nprob=3, nmin=100, nmax=300, occ_min=0.02, occ_max=0.08)
    mats, plans = [], []
    for p in probs:
        A, B = to_lib(p.A), to_lib(p.B)
        pl = bst.multiply_plan(A, B, None, p.eps)
        pl.alloc_result()
        mats.append((A, B))
        plans.append(pl)
    batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
    n = len(plans)
    bst.bst_batch_execute(batch, np.ones(n), np.zeros(n), prec)  # first (untimed) run
    torch.cuda.synchronize()
    torch.cuda._sleep(200_000_000)  # keeps the stream busy for ~0.1 s
    bst.bst_batch_execute(batch, np.full(n, 2.0), np.zeros(n), prec)
    first = [pl.result.data[:pl.result.info[3]].clone() for pl in plans]
    bst.bst_batch_execute(batch, np.full(n, -3.0), np.zeros(n), prec)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == bst.BST_FP64 else 1e-11
    for q, p in enumerate(probs):
        ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)["data"]
        assert rel_fro(first[q].cpu().numpy(), 2.0 * ref) <= tol
        second = plans[q].result.data[:plans[q].result.info[3]].cpu().numpy()
        assert rel_fro(second, -3.0 * ref) <= tol
    bst.bst_batch_destroy(batch)
