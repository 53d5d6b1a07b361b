"""GPU adjoint (sampled block-sparse products) against the CPU oracle's adjoint, the
dot-product identity, central finite differences and torch.autograd."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from helpers import random_matrix, transpose_matrix
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import Problem, banded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _mixed(seed, nb=(25, 30, 20), occ=0.2, sizes=(5, 13, 23), ta="N", tb="N", cin=True):
    rng = np.random.default_rng(seed)
    s = np.asarray(sizes, np.int32)
    m, k, n = (rng.choice(s, c).astype(np.int32) for c in nb)
    A = random_matrix(rng, m, k, occ)
    B = random_matrix(rng, k, n, occ)
    Ci = random_matrix(rng, m, n, occ) if cin else None
    if ta == "T":
        A = transpose_matrix(A)
    if tb == "T":
        B = transpose_matrix(B)
    return Problem(A, B, Ci, 1.25, -0.5, 0.0, ta, tb)


def gpu_adjoint(p, G):
    import torch
    A, B = to_lib(p.A), to_lib(p.B)
    Ci = to_lib(p.C_in) if p.C_in is not None else None
    plan = bst.multiply(A, B, Ci, p.alpha, p.beta, p.eps, p.transa, p.transb)
    g = torch.as_tensor(G).cuda()
    dA = torch.full_like(A.data, np.nan)
    dB = torch.full_like(B.data, np.nan)
    dCi = torch.full_like(Ci.data, np.nan) if Ci is not None else None
    bst.bst_plan_adjoint(plan.handle, g, dA, dB, dCi, p.alpha, p.beta)
    torch.cuda.synchronize()
    return (dA.cpu().numpy(), dB.cpu().numpy(), None if dCi is None else dCi.cpu().numpy(),
            plan)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_adjoint_vs_oracle(ta, tb):
    p = _mixed(1, ta=ta, tb=tb)
    ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, ta, tb)
    G = np.random.default_rng(2).standard_normal(len(ref["data"]))
    rA, rB, rC = oracle.multiply_adjoint(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, G, ta, tb)
    dA, dB, dC, _ = gpu_adjoint(p, G)
    assert rel_fro(dA, rA) <= 1e-12 and rel_fro(dB, rB) <= 1e-12
    assert (dC == rC).all()


def test_adjoint_with_filter_and_generic_sizes():
    p = banded(seed=3, nb=300, decay=40.0, value_decay=8.0, eps=1e-8)
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    assert ref["nfiltered"] > 0
    G = ref["data"].copy()
    rA, rB, _ = oracle.multiply_adjoint(p.A, p.B, None, 1.0, 0.0, p.eps, G)
    dA, dB, _, _ = gpu_adjoint(p, G)
    assert rel_fro(dA, rA) <= 1e-12 and rel_fro(dB, rB) <= 1e-12
    p2 = _mixed(4, nb=(7, 9, 6), occ=0.4, sizes=(1, 3, 31, 40))
    ref = oracle.multiply(p2.A, p2.B, p2.C_in, p2.alpha, p2.beta)
    G = np.random.default_rng(5).standard_normal(len(ref["data"]))
    rA, rB, rC = oracle.multiply_adjoint(p2.A, p2.B, p2.C_in, p2.alpha, p2.beta, 0.0, G)
    dA, dB, dC, _ = gpu_adjoint(p2, G)
    assert rel_fro(dA, rA) <= 1e-12 and rel_fro(dB, rB) <= 1e-12


def test_autograd_matches_adjoint_and_fd():
    import torch
    from paper_1910_13555_gb300 import autograd
    p = _mixed(6, cin=False)
    A, B = to_lib(p.A), to_lib(p.B)
    A.data.requires_grad_(True)
    B.data.requires_grad_(True)
    c, plan = autograd.multiply(A, B, None, 1.0, 0.0)
    nel = bst.bst_matrix_info(bst.bst_plan_result(plan.handle))[3]
    loss = 0.5 * (c[:nel] ** 2).sum()
    loss.backward()
    ref = oracle.multiply(p.A, p.B)
    rA, rB, _ = oracle.multiply_adjoint(p.A, p.B, None, 1.0, 0.0, 0.0, ref["data"])
    assert rel_fro(A.data.grad.cpu().numpy(), rA) <= 1e-12
    assert rel_fro(B.data.grad.cpu().numpy(), rB) <= 1e-12
    # central differences on the GPU path (the loss is quadratic in each entry)
    h = 1e-6
    L = float(loss)
    rng = np.random.default_rng(7)
    with torch.no_grad():
        for M, g in ((A, A.data.grad), (B, B.data.grad)):
            for e in rng.choice(M.data.numel(), 10, replace=False):
                old = float(M.data[e])
                M.data[e] = old + h
                lp = 0.5 * float((bst.multiply(A, B).result.data[:nel] ** 2).sum())
                M.data[e] = old - h
                lm = 0.5 * float((bst.multiply(A, B).result.data[:nel] ** 2).sum())
                M.data[e] = old
                fd = (lp - lm) / (2 * h)
                gv = float(g[e])
                assert abs(fd - gv) <= 1e-7 * max(1, abs(gv)) + 8 * 2.0 ** -52 * L / h


def test_multiply_adjoint_equals_plan_adjoint_without_cin():
    import torch
    p = _mixed(41, cin=False)
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply(A, B, None, p.alpha, 0.0, p.eps, p.transa, p.transb)
    assert bst.bst_matrix_data_size(plan.result.handle) == plan.result.info[3]
    assert bst.bst_matrix_data_size(A.handle) == len(p.A.data)
    g = torch.randn(plan.result.info[3], dtype=torch.float64, device="cuda")
    dA1, dB1 = torch.empty_like(A.data), torch.empty_like(B.data)
    dA2, dB2 = torch.empty_like(A.data), torch.empty_like(B.data)
    bst.bst_plan_adjoint(plan.handle, g, dA1, dB1, None, p.alpha, 0.0)
    bst.bst_multiply_adjoint(plan.handle, g, dA2, dB2, p.alpha)
    torch.cuda.synchronize()
    assert torch.equal(dA1, dA2) and torch.equal(dB1, dB2)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_adjoint_tall_b_blocks(ta, tb):
    """op(B) blocks of 20, 70 and 130 rows with 5 to 40 columns (outputs spread over
    several warps): every layout against the oracle's adjoint, repeat runs bitwise
    equal."""
    rng = np.random.default_rng(7)
    m = rng.choice(np.array([5, 13], np.int32), 12).astype(np.int32)
    k = rng.choice(np.array([20, 70, 130], np.int32), 10).astype(np.int32)
    n = rng.choice(np.array([5, 13, 40], np.int32), 9).astype(np.int32)
    A = random_matrix(rng, m, k, 0.4)
    B = random_matrix(rng, k, n, 0.4)
    Ci = random_matrix(rng, m, n, 0.3)
    if ta == "T":
        A = transpose_matrix(A)
    if tb == "T":
        B = transpose_matrix(B)
    p = Problem(A, B, Ci, 0.75, 2.0, 0.0, ta, tb)
    ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, ta, tb)
    G = rng.standard_normal(len(ref["data"]))
    rA, rB, rC = oracle.multiply_adjoint(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, G, ta, tb)
    dA, dB, dC, _ = gpu_adjoint(p, G)
    assert rel_fro(dA, rA) <= 1e-12 and rel_fro(dB, rB) <= 1e-12
    assert (dC == rC).all()
    dA2, dB2, _, _ = gpu_adjoint(p, G)
    assert (dB2 == dB).all() and (dA2 == dA).all()
