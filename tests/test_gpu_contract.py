"""GPU block-sparse tensor contraction (remap to matrices + multiply, paper Sec. 4)
against the CPU oracle's contraction: result block index bit-exact, values within
1e-12 (FP64) / 1e-11 (emulated FP64); adjoint against the oracle's adjoint."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import random_tensor, rank3

pytestmark = pytest.mark.gpu

SZ = np.array([2, 3, 5, 13], np.int32)

CASES = [
    (3, 3, [2], [0], [0, 1], [1, 2], None),          # zero-copy A and B
    (3, 3, [0, 2], [0, 1], [1], [2], None),          # rank-3 workload: A permuted
    (3, 3, [0, 2], [0, 1], [1], [2], [1, 0]),        # ... and the result permuted
    (4, 3, [1, 3], [2, 0], [0, 2], [1], [2, 0, 1]),
    (4, 4, [0, 1, 2], [3, 1, 0], [3], [2], [1, 0]),  # three index pairs
    (2, 2, [0], [0], [1], [1], None),                # A^T B (zero-copy transpose)
    (3, 3, [0], [2], [1, 2], [0, 1], None),          # zero-copy transposes on both sides
    (4, 2, [3], [0], [0, 1, 2], [1], [3, 1, 0, 2]),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _make(seed, case, occ=0.5):
    r1, r2, c1, c2, f1, f2, ro = case
    rng = np.random.default_rng(seed)
    nb1 = [int(rng.integers(2, 5)) for _ in range(r1)]
    s1 = [rng.choice(SZ, n).astype(np.int32) for n in nb1]
    nb2 = [0] * r2
    s2 = [None] * r2
    for a, b in zip(c1, c2):
        nb2[b] = nb1[a]
        s2[b] = s1[a]
    for b in f2:
        nb2[b] = int(rng.integers(2, 5))
        s2[b] = rng.choice(SZ, nb2[b]).astype(np.int32)
    return random_tensor(rng, nb1, s1, occ), random_tensor(rng, nb2, s2, occ)


def _rsizes(T1, T2, case):
    _, _, c1, c2, f1, f2, ro = case
    free = [T1.block_sizes[a] for a in f1] + [T2.block_sizes[b] for b in f2]
    ro = ro if ro is not None else list(range(len(free)))
    return [free[r] for r in ro]


def gpu_contract(T1, T2, case, R_in=None, alpha=1.0, beta=0.0, eps=0.0, prec=bst.BST_FP64):
    import torch
    _, _, c1, c2, f1, f2, ro = case
    t1 = bst.Tensor.from_host(T1.block_sizes, T1.index, T1.data)
    t2 = bst.Tensor.from_host(T2.block_sizes, T2.index, T2.data)
    ri = bst.Tensor.from_host(R_in.block_sizes, R_in.index, R_in.data) if R_in is not None else None
    plan = bst.contract(t1, t2, c1, c2, f1, f2, ro, ri, alpha, beta, eps, prec)
    torch.cuda.synchronize()
    idx, off = plan.result.index()
    ne = plan.result.info[2]
    return idx, off, plan.result.data[:ne].cpu().numpy(), plan, (t1, t2, ri)


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("prec", [bst.BST_FP64, bst.BST_FP64_EMU_BF16])
def test_contract_vs_oracle(ci, prec):
    case = CASES[ci]
    _, _, c1, c2, f1, f2, ro = case
    T1, T2 = _make(ci, case)
    rs = _rsizes(T1, T2, case)
    rng = np.random.default_rng(100 + ci)
    Rin = random_tensor(rng, [len(s) for s in rs], rs, 0.4)
    ref = oracle.contract(T1, T2, c1, c2, f1, f2, ro, Rin, 0.75, -1.5, 0.0)
    idx, off, data, _, _ = gpu_contract(T1, T2, case, Rin, 0.75, -1.5, 0.0, prec)
    assert (idx == ref["index"]).all() and (off == ref["offsets"]).all()
    tol = 1e-12 if prec == bst.BST_FP64 else 1e-11
    assert rel_fro(data, ref["data"]) <= tol


def test_contract_filter():
    case = CASES[1]
    _, _, c1, c2, f1, f2, ro = case
    T1, T2 = _make(77, case, occ=0.7)
    rng = np.random.default_rng(5)
    T1.data *= np.repeat(10.0 ** -rng.uniform(0, 3, T1.nblocks), T1.block_lens)
    full = oracle.contract(T1, T2, c1, c2, f1, f2, ro)
    eps = 0.3 * float(np.median(np.abs(full["data"]))) + 1e-3
    ref = oracle.contract(T1, T2, c1, c2, f1, f2, ro, None, 1.0, 0.0, eps)
    idx, off, data, plan, _ = gpu_contract(T1, T2, case, eps=eps)
    assert (idx == ref["index"]).all()
    assert plan.stats()["n_stack"] == ref["npairs"]
    assert rel_fro(data, ref["data"]) <= 1e-12


def test_rank3_workload_small_and_adjoint():
    import torch
    w = rank3(seed=9, nP=40, sP=30, nao=30, window=6, p=0.4)
    ref = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    case = (3, 3, w.c1, w.c2, w.f1, w.f2, w.result_order)
    idx, off, data, plan, (t1, t2, _) = gpu_contract(w.T1, w.T2, case)
    assert (idx == ref["index"]).all()
    assert rel_fro(data, ref["data"]) <= 1e-12
    # loss = 1/2 ||R||^2: dR = R
    rT, rU, _ = oracle.contract_adjoint(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order,
                                         None, 1.0, 0.0, 0.0, ref["data"])
    dR = plan.result.data
    dT = torch.full_like(t1.data, np.nan)
    dU = torch.full_like(t2.data, np.nan)
    bst.bst_plan_adjoint(plan.handle, dR, dT, dU, None, 1.0, 0.0)
    torch.cuda.synchronize()
    assert rel_fro(dT.cpu().numpy(), rT) <= 1e-12
    assert rel_fro(dU.cpu().numpy(), rU) <= 1e-12


@pytest.mark.parametrize("ci", [2, 3, 4])
def test_contract_adjoint_permuted(ci):
    import torch
    case = CASES[ci]
    _, _, c1, c2, f1, f2, ro = case
    T1, T2 = _make(300 + ci, case)
    rs = _rsizes(T1, T2, case)
    Rin = random_tensor(np.random.default_rng(ci), [len(s) for s in rs], rs, 0.4)
    ref = oracle.contract(T1, T2, c1, c2, f1, f2, ro, Rin, 1.25, 0.5, 0.0)
    G = np.random.default_rng(1).standard_normal(len(ref["data"]))
    r1, r2, rri = oracle.contract_adjoint(T1, T2, c1, c2, f1, f2, ro, Rin, 1.25, 0.5, 0.0, G)
    idx, off, data, plan, (t1, t2, ri) = gpu_contract(T1, T2, case, Rin, 1.25, 0.5)
    g = torch.as_tensor(G).cuda()
    d1 = torch.full_like(t1.data, np.nan)
    d2 = torch.full_like(t2.data, np.nan)
    dri = torch.full_like(ri.data, np.nan)
    bst.bst_plan_adjoint(plan.handle, g, d1, d2, dri, 1.25, 0.5)
    torch.cuda.synchronize()
    assert rel_fro(d1.cpu().numpy(), r1) <= 1e-12
    assert rel_fro(d2.cpu().numpy(), r2) <= 1e-12
    assert rel_fro(dri.cpu().numpy(), rri) <= 1e-15
