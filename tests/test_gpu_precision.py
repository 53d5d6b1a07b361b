"""GPU parity of the emulated-FP64 (BF16 Ozaki slices) and 3xTF32 paths against the CPU
oracle: same plan, so patterns and stacks are those of the FP64 tests; values within
1e-11 (emulated FP64) and 1e-5 (3xTF32) relative Frobenius error."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, run_multiply
from helpers import random_matrix, transpose_matrix
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import Problem, banded, batched, tall_skinny

pytestmark = pytest.mark.gpu

TOL = {bst.BST_FP64_EMU_BF16: 1e-11, bst.BST_TF32X3: 1e-5}
PRECS = [bst.BST_FP64_EMU_BF16, bst.BST_TF32X3]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def check(p, prec):
    ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, p.transa, p.transb)
    got = run_multiply(p, precision=prec, stacks=False)
    assert (got["rows"] == ref["rows"]).all() and (got["cols"] == ref["cols"]).all()
    err = rel_fro(got["data"], ref["data"])
    assert err <= TOL[prec], err
    return err


def _mixed(seed, nb=(30, 40, 35), occ=0.15, sizes=(5, 13, 23), cin=True, alpha=1.0, beta=0.0,
           ta="N", tb="N", scale_decades=0.0, dist="uniform"):
    rng = np.random.default_rng(seed)
    s = np.asarray(sizes, np.int32)
    m, k, n = (rng.choice(s, c).astype(np.int32) for c in nb)
    A = random_matrix(rng, m, k, occ, dist)
    B = random_matrix(rng, k, n, occ, dist)
    if scale_decades:
        A.data *= np.repeat(10.0 ** -rng.uniform(0, scale_decades, A.nblocks), A.block_lens)
        B.data *= np.repeat(10.0 ** -rng.uniform(0, scale_decades, B.nblocks), B.block_lens)
    Ci = random_matrix(rng, m, n, occ) if cin else None
    if ta == "T":
        A = transpose_matrix(A)
    if tb == "T":
        B = transpose_matrix(B)
    return Problem(A, B, Ci, alpha, beta, 0.0, ta, tb)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_mixed_transposes(prec, ta, tb):
    check(_mixed(1, ta=ta, tb=tb, alpha=-0.5, beta=2.0), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_generic_and_large_blocks(prec):
    # m, n > 16 in several tiles, k > 160 (several exact FP32 segments), sizes 1 and odd
    check(_mixed(2, nb=(9, 7, 8), occ=0.4, sizes=(1, 7, 31, 40, 170), alpha=1.5, beta=0.5), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_banded_with_filter(prec):
    check(banded(seed=3, nb=300, decay=40.0, value_decay=8.0, eps=1e-8), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_tall_skinny(prec):
    check(tall_skinny(seed=4, nk=3000, nmn=48, window=10, p=0.3), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_wide_dynamic_range(prec):
    # per-block scales over 8 decades (the batched workload's recipe), normal entries
    check(_mixed(5, scale_decades=8.0, dist="normal", cin=False), prec)


def test_batched_problem_emulated():
    p = batched(nprob=3, nmin=200, nmax=400, occ_min=0.02, occ_max=0.05)[1]
    check(p, bst.BST_FP64_EMU_BF16)


def test_emulated_deterministic_and_zero_blocks():
    p = _mixed(6, cin=False)
    # a few all-zero blocks and rows
    p.A.data[:p.A.block_lens[0]] = 0.0
    a = run_multiply(p, precision=bst.BST_FP64_EMU_BF16, stacks=False)
    b = run_multiply(p, precision=bst.BST_FP64_EMU_BF16, stacks=False)
    assert (a["data"] == b["data"]).all()
    ref = oracle.multiply(p.A, p.B)
    assert rel_fro(a["data"], ref["data"]) <= 1e-11


def test_integer_data_exact():
    """Small integers: every digit product and sum is exact, so the emulated result
    equals the exact product bit for bit."""
    rng = np.random.default_rng(7)
    p = _mixed(7, cin=False)
    p.A.data[:] = rng.integers(-50, 51, len(p.A.data))
    p.B.data[:] = rng.integers(-50, 51, len(p.B.data))
    ref = oracle.multiply(p.A, p.B)
    got = run_multiply(p, precision=bst.BST_FP64_EMU_BF16, stacks=False)
    assert (got["data"] == ref["data"]).all()


@pytest.mark.parametrize("case", ["transposed", "wide_range", "large_blocks", "tall_skinny"])
def test_emulated_block_scaled(case):
    """The block-scaled digit mode (exponents per block row / column instead of per whole
    op row / column) meets the same bound."""
    ctx = bst.context()
    old = bst.bst_tune_get(ctx, bst.BST_TUNE_EMU_ROW_SCALE)
    bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_ROW_SCALE, 0)
    try:
        p = {"transposed": lambda: _mixed(11, ta="T", tb="T", alpha=-0.5, beta=2.0),
             "wide_range": lambda: _mixed(12, scale_decades=8.0, dist="normal", cin=False),
             "large_blocks": lambda: _mixed(13, nb=(9, 7, 8), occ=0.4, sizes=(1, 7, 31, 40, 170)),
             "tall_skinny": lambda: tall_skinny(seed=14, nk=3000, nmn=48, window=10, p=0.3)}[case]()
        check(p, bst.BST_FP64_EMU_BF16)
    finally:
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_ROW_SCALE, old)


def test_emulated_many_products_per_block():
    """C blocks with far more than 32 products (the entry list is walked 32 at a time)."""
    p = tall_skinny(seed=15, nk=4000, nmn=8, window=8, p=0.5)
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb)
    st = run_multiply(p, precision=bst.BST_FP64, stacks=True)
    _, per_block = np.unique(st["c_off"], return_counts=True)
    assert per_block.max() > 64
    got = run_multiply(p, precision=bst.BST_FP64_EMU_BF16, stacks=False)
    assert rel_fro(got["data"], ref["data"]) <= 1e-11


def test_emulated_long_inner_sums_alone_and_batched():
    """Plans whose C elements sum at least 64 inner elements on average take the
    pipelined row-scaled tile loop, alone and in a batch: within 1e-11 of the oracle,
    and the batch equal to the single executes bit for bit."""
    import torch

    from gpu_util import to_lib
    probs = [tall_skinny(seed=40 + q, nk=3000, nmn=12, window=6, p=0.5) for q in range(2)]
    mats, plans, refs = [], [], []
    for p in probs:
        A, B = to_lib(p.A), to_lib(p.B)
        pl = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
        pl.alloc_result()
        assert pl.stats()["flops"] >= 2 * 64 * pl.result.info[3]
        mats.append((A, B))
        plans.append(pl)
        refs.append(oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb))
    single = []
    for pl, ref in zip(plans, refs):
        pl.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
        got = pl.result.data[:pl.result.info[3]].cpu().numpy().copy()
        assert rel_fro(got, ref["data"]) <= 1e-11
        single.append(got)
    batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
    bst.bst_batch_execute(batch, np.ones(2), np.zeros(2), bst.BST_FP64_EMU_BF16)
    torch.cuda.synchronize()
    for pl, s in zip(plans, single):
        assert (pl.result.data[:pl.result.info[3]].cpu().numpy() == s).all()
    bst.bst_batch_destroy(batch)
