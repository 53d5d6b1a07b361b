"""Full-size workloads on the GPU, checked on sampled output blocks against the CPU
oracle (which computes exactly the sampled blocks from the definition) and against
properties that hold at any size: the tall-skinny A^T B with split-K, the rank-3
contraction forward + adjoint (dot-product identity and central differences on 50
sampled entries), and the 64-problem batch in one persistent launch."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import batched, rank3, tall_skinny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _gather(data, offs, lens):
    import torch
    idx = np.concatenate([np.arange(o, o + n) for o, n in zip(offs, lens)])
    return data[torch.as_tensor(idx, device=data.device)].cpu().numpy()


def test_tall_skinny_full_size_split_k():
    import torch
    p = tall_skinny()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    rows, cols, offs = C.index()
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(rows), 64, replace=False))
    ref, present = oracle.multiply_sample(p.A, p.B, None, 1.0, 0.0, p.eps, rows[sel], cols[sel],
                                          transa="T", row_sizes=p.A.col_sizes,
                                          col_sizes=p.B.col_sizes)
    assert present.all()
    lens = p.A.col_sizes[rows[sel]].astype(np.int64) * p.B.col_sizes[cols[sel]]
    out = {}
    for split in (1, 4, 0):
        plan.execute(1.0, 0.0, bst.BST_FP64, split)
        torch.cuda.synchronize()
        out[split] = C.data[:C.info[3]].clone()
        assert rel_fro(_gather(C.data, offs[sel], lens), ref) <= 1e-12
    assert float((out[4] - out[1]).norm() / out[1].norm()) <= 1e-14
    plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
    torch.cuda.synchronize()
    assert rel_fro(_gather(C.data, offs[sel], lens), ref) <= 1e-11
    # stack count = sum over K row blocks of nnz(A row) * nnz(B row)
    ra = np.bincount(p.A.rows, minlength=len(p.A.row_sizes)).astype(np.int64)
    rb = np.bincount(p.B.rows, minlength=len(p.B.row_sizes)).astype(np.int64)
    assert plan.stats()["n_stack"] == int((ra * rb).sum())


def test_rank3_full_size_forward_adjoint_fd():
    import torch
    w = rank3()
    t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data)
    t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data)
    plan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    torch.cuda.synchronize()
    R = plan.result
    idx, offs = R.index()
    rs = [w.T1.block_sizes[1], w.T2.block_sizes[2]]
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(len(idx), 32, replace=False))
    ref, present = oracle.contract_sample(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order,
                                          None, 1.0, 0.0, 0.0, idx[sel], rs)
    assert present.all()
    lens = rs[0][idx[sel, 0]].astype(np.int64) * rs[1][idx[sel, 1]]
    assert rel_fro(_gather(R.data, offs[sel], lens), ref) <= 1e-12
    # adjoint of L = 1/2 ||R||^2: dR = R; bilinearity gives <dT, T> = <dU, U> = ||R||^2
    ne = R.info[2]
    dR = R.data[:ne].clone()
    dT = torch.empty_like(t1.data)
    dU = torch.empty_like(t2.data)
    bst.bst_plan_adjoint(plan.handle, dR, dT, dU, None, 1.0, 0.0)
    torch.cuda.synchronize()
    rr = float((dR * dR).sum())
    assert abs(float((dT * t1.data).sum()) - rr) <= 1e-12 * rr
    assert abs(float((dU * t2.data).sum()) - rr) <= 1e-12 * rr
    # central differences on 25 entries of T and 25 of U (the loss is quadratic in each)
    h = 1e-6
    L = 0.5 * rr

    def loss():
        plan.execute(1.0, 0.0, bst.BST_FP64, 1)
        return 0.5 * float((R.data[:ne] ** 2).sum())

    for M, g in ((t1, dT), (t2, dU)):
        for e in rng.choice(M.data.numel(), 25, replace=False):
            old = float(M.data[e])
            M.data[e] = old + h
            lp = loss()
            M.data[e] = old - h
            lm = loss()
            M.data[e] = old
            fd = (lp - lm) / (2 * h)
            gv = float(g[e])
            assert abs(fd - gv) <= 1e-7 * max(1.0, abs(gv)) + 8 * 2.0 ** -52 * L / h


def test_batched_full_size_one_launch():
    import torch
    probs = batched()
    mats, plans = [], []
    for p in probs:
        A, B = to_lib(p.A), to_lib(p.B)
        plan = bst.multiply_plan(A, B, None, p.eps)
        plan.alloc_result()
        mats.append((A, B))
        plans.append(plan)
    batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
    rng = np.random.default_rng(2)
    for prec, tol in ((bst.BST_FP64, 1e-12), (bst.BST_FP64_EMU_BF16, 1e-11)):
        bst.bst_batch_execute(batch, np.ones(len(plans)), np.zeros(len(plans)), prec)
        torch.cuda.synchronize()
        for q in rng.choice(len(probs), 8, replace=False):
            p, pl = probs[q], plans[q]
            rows, cols, offs = pl.result.index()
            if len(rows) == 0:
                continue
            sel = np.sort(rng.choice(len(rows), min(16, len(rows)), replace=False))
            ref, _ = oracle.multiply_sample(p.A, p.B, None, 1.0, 0.0, p.eps, rows[sel], cols[sel],
                                            row_sizes=p.A.row_sizes, col_sizes=p.B.col_sizes)
            lens = p.A.row_sizes[rows[sel]].astype(np.int64) * p.B.col_sizes[cols[sel]]
            assert rel_fro(_gather(pl.result.data, offs[sel], lens), ref) <= tol
    bst.bst_batch_destroy(batch)
