"""Slab reading of a contraction operand (the second remap of T(P, mu, nu) contracted over
(P, nu): its matrix view rows = mu, columns = (P, nu) is read in place as P consecutive
mu x nu slabs of each tensor block instead of through a permuted copy): native FP64
with and without it, the other precisions, split-K, the adjoint and batches all match
the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import _tensor, rank3

pytestmark = pytest.mark.gpu

TOL = {bst.BST_FP64: 1e-12, bst.BST_FP64_EMU_BF16: 1e-11, bst.BST_TF32X3: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture()
def ctx():
    c = bst.context()
    prev = bst.bst_tune_get(c, bst.BST_TUNE_CONTRACT_SLAB)
    yield c
    bst.bst_tune_set(c, bst.BST_TUNE_CONTRACT_SLAB, prev)


def _lib(T):
    return bst.Tensor.from_host(T.block_sizes, T.index, T.data)


def _plan(ctx, w, slab, R_in=None):
    bst.bst_tune_set(ctx, bst.BST_TUNE_CONTRACT_SLAB, slab)
    t1, t2 = _lib(w.T1), _lib(w.T2)
    ri = _lib(R_in) if R_in is not None else None
    plan = bst.contract_plan(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, ri, 0.0)
    plan.alloc_result()
    return plan, (t1, t2, ri)


def _result(plan):
    import torch
    torch.cuda.synchronize()
    idx, off = plan.result.index()
    return idx, plan.result.data[:plan.result.info[2]].cpu().numpy()


def _wide_slabs(seed=5):
    """T(P, mu, nu) with nu = 60 (slabs wider than a 13 x 13 panel of 59) beside nu = 5."""
    rng = np.random.default_rng(seed)
    nP, nao = 12, 10
    psz = np.full(nP, 3, np.int32)
    musz = rng.choice(np.array([5, 13], np.int32), nao).astype(np.int32)
    nusz = np.where(np.arange(nao) % 2 == 0, 60, 5).astype(np.int32)
    keep = rng.random((nP, nao, nao)) < 0.3
    T = _tensor(rng, [psz, musz, nusz], np.stack(np.nonzero(keep), 1))
    keep = rng.random((nP, nao, nao)) < 0.3
    U = _tensor(rng, [psz, nusz, musz], np.stack(np.nonzero(keep), 1))
    return T, U


class _W:
    def __init__(self, T1, T2, c1=(0, 2), c2=(0, 1), f1=(1,), f2=(2,), ro=None):
        self.T1, self.T2 = T1, T2
        self.c1, self.c2, self.f1, self.f2 = list(c1), list(c2), list(f1), list(f2)
        self.result_order = ro


def _rank3_small(seed=11):
    return rank3(seed=seed, nP=50, sP=30, nao=36, window=6, p=0.4)


@pytest.mark.parametrize("slab", [0, 1])
@pytest.mark.parametrize("prec", [bst.BST_FP64, bst.BST_FP64_EMU_BF16, bst.BST_TF32X3])
def test_rank3_with_and_without_slabs(ctx, slab, prec):
    w = _rank3_small()
    rng = np.random.default_rng(3)
    ref0 = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    # a result-pattern R_in (every other block of the plain result, random values)
    keep = np.arange(len(ref0["index"])) % 2 == 0
    rs = [w.T1.block_sizes[1], w.T2.block_sizes[2]]
    R_in = _tensor(rng, rs, ref0["index"][keep])
    ref = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order, R_in, 0.5, -2.0)
    plan, keep_ = _plan(ctx, w, slab, R_in)
    assert plan.schedule_info()["slab"] == bool(slab)
    plan.execute(0.5, -2.0, prec, 1)
    idx, data = _result(plan)
    assert (idx == ref["index"]).all()
    assert rel_fro(data, ref["data"]) <= TOL[prec]


def test_slabs_wider_than_a_panel(ctx):
    T, U = _wide_slabs()
    w = _W(T, U)
    ref = oracle.contract(T, U, w.c1, w.c2, w.f1, w.f2, None)
    for slab in (1, 0):
        plan, keep = _plan(ctx, w, slab)
        assert plan.schedule_info()["slab"] == bool(slab)
        plan.execute(1.0, 0.0, bst.BST_FP64, 1)
        idx, data = _result(plan)
        assert (idx == ref["index"]).all()
        assert rel_fro(data, ref["data"]) <= 1e-12


def test_mixed_slab_widths_fall_back_to_the_copy(ctx):
    # P sizes {2, 13} and nu sizes {13, 2}: a 26-wide k block is 2 slabs of 13 or 13 of 2
    rng = np.random.default_rng(8)
    psz = rng.choice(np.array([2, 13], np.int32), 10).astype(np.int32)
    musz = rng.choice(np.array([5, 13], np.int32), 8).astype(np.int32)
    nusz = rng.choice(np.array([2, 13], np.int32), 8).astype(np.int32)
    T = _tensor(rng, [psz, musz, nusz], np.stack(np.nonzero(rng.random((10, 8, 8)) < 0.4), 1))
    U = _tensor(rng, [psz, nusz, musz], np.stack(np.nonzero(rng.random((10, 8, 8)) < 0.4), 1))
    w = _W(T, U)
    ref = oracle.contract(T, U, w.c1, w.c2, w.f1, w.f2, None)
    plan, keep = _plan(ctx, w, 1)
    assert not plan.schedule_info()["slab"]
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    idx, data = _result(plan)
    assert (idx == ref["index"]).all()
    assert rel_fro(data, ref["data"]) <= 1e-12


def test_slab_plan_split_k_and_adjoint(ctx):
    import torch
    w = _rank3_small(seed=12)
    ref = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    plan, (t1, t2, _) = _plan(ctx, w, 1)
    assert plan.schedule_info()["slab"]
    plan.execute(1.0, 0.0, bst.BST_FP64, 3)  # the K split reads the slabs in place too
    idx, data = _result(plan)
    assert rel_fro(data, ref["data"]) <= 1e-12
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    idx, data = _result(plan)
    assert rel_fro(data, ref["data"]) <= 1e-12
    G = np.random.default_rng(2).standard_normal(len(ref["data"]))
    rT, rU, _ = oracle.contract_adjoint(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order,
                                         None, 1.0, 0.0, 0.0, G)
    dT = torch.full_like(t1.data, np.nan)
    dU = torch.full_like(t2.data, np.nan)
    bst.bst_plan_adjoint(plan.handle, torch.as_tensor(G).cuda(), dT, dU, None, 1.0, 0.0)
    torch.cuda.synchronize()
    assert rel_fro(dT.cpu().numpy(), rT) <= 1e-12
    assert rel_fro(dU.cpu().numpy(), rU) <= 1e-12
    # after the adjoint (which permuted the copy) the in-place forward still matches
    t1.data.mul_(-1.0)
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    idx, data = _result(plan)
    assert rel_fro(data, -ref["data"]) <= 1e-12


def test_slab_plan_in_a_batch(ctx):
    from gpu_util import to_lib
    from paper_1910_13555_gb300.workloads import banded
    w = _rank3_small(seed=13)
    ref = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    plan, keep = _plan(ctx, w, 1)
    assert plan.schedule_info()["slab"]
    p = banded(seed=14, nb=120, decay=20.0, value_decay=8.0, eps=0.0)
    A, B = to_lib(p.A), to_lib(p.B)
    mp = bst.multiply_plan(A, B, None, 0.0)
    C = mp.alloc_result()
    batch = bst.bst_batch_create(ctx, [plan.handle, mp.handle])
    bst.bst_batch_execute(batch, [1.0, 1.0], [0.0, 0.0], bst.BST_FP64)
    idx, data = _result(plan)
    assert rel_fro(data, ref["data"]) <= 1e-12
    r = oracle.multiply(p.A, p.B, None, 1.0, 0.0, 0.0)
    assert rel_fro(C.data[:C.info[3]].cpu().numpy(), r["data"]) <= 1e-12
    bst.bst_batch_destroy(batch)


def test_tuner_picks_a_remap(ctx):
    from paper_1910_13555_gb300 import tune
    w = _rank3_small(seed=15)
    t1, t2 = _lib(w.T1), _lib(w.T2)
    res = tune.tune_contract_slab(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, reps=2)
    assert res["slab"] in (0, 1) and res["ms"][res["slab"]] == min(res["ms"].values())
    assert bst.bst_tune_get(ctx, bst.BST_TUNE_CONTRACT_SLAB) == res["slab"]
    assert set(res["eligible"].values()) == {True}
