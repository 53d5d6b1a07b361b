"""GPU parity of the block-sparse multiply against the CPU oracle, through the C ABI.

Patterns, stacks and offsets must match bit for bit; values within 1e-12 relative
Frobenius error (native FP64).  Cases span several (m,n,k) buckets, transposes,
alpha/beta with C_in, the norm filter, empty and degenerate inputs, split-K and
determinism.  The full-size banded workload is checked on sampled blocks.
"""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, run_multiply
from helpers import random_matrix, transpose_matrix
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import BSMatrix, Problem, banded, plain, tall_skinny

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def check_parity(p, split_k=1, stacks=True, tol=TOL_FP64):
    ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, p.transa, p.transb)
    got = run_multiply(p, split_k=split_k, stacks=stacks)
    assert (got["rows"] == ref["rows"]).all() and (got["cols"] == ref["cols"]).all()
    assert (got["offsets"] == ref["offsets"]).all()
    st = got["stats"]
    assert st["n_stack"] == len(ref["a_off"])
    assert st["n_filtered"] == ref["nfiltered"]
    assert st["n_candidates"] == ref["ncandidates"]
    assert st["flops"] == ref["flops"]
    if stacks:
        assert (got["mnk"] == ref["mnk"]).all()
        assert (got["bucket_ptr"] == ref["bucket_ptr"]).all()
        assert (got["a_off"] == ref["a_off"]).all()
        assert (got["b_off"] == ref["b_off"]).all()
        assert (got["c_off"] == ref["c_off"]).all()
    err = rel_fro(got["data"], ref["data"])
    assert err <= tol, err
    return got, ref


def _mixed(seed, nb=(30, 40, 35), occ=0.15, sizes=(5, 13, 23), cin=True, alpha=1.0, beta=0.0,
           eps=0.0, ta="N", tb="N"):
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
    return Problem(A, B, Ci, alpha, beta, eps, ta, tb)


def test_plain_workload():
    check_parity(plain())


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_mixed_sizes_transposes_alpha_beta(ta, tb):
    check_parity(_mixed(1, ta=ta, tb=tb, alpha=-0.5, beta=2.0))


def test_generic_sizes_and_ragged_rows():
    # sizes outside the specialised set (generic path), one large block (> 256 outputs)
    check_parity(_mixed(2, nb=(17, 19, 21), occ=0.3, sizes=(1, 2, 7, 31, 40), alpha=1.5, beta=0.5))


def test_banded_with_filter():
    # same recipe at 300 blocks with shorter decay lengths so that the filter bites
    p = banded(seed=3, nb=300, decay=40.0, value_decay=8.0, eps=1e-8)
    got, ref = check_parity(p)
    assert ref["nfiltered"] > 0


def test_tall_skinny_transposed():
    check_parity(tall_skinny(seed=4, nk=3000, nmn=48, window=10, p=0.3))


@pytest.mark.parametrize("split", [2, 3, 8])
def test_split_k_equals_unsplit(split):
    p = tall_skinny(seed=5, nk=4000, nmn=40, window=8, p=0.4)
    one = run_multiply(p, split_k=1, stacks=False)
    many = run_multiply(p, split_k=split, stacks=False)
    assert (one["rows"] == many["rows"]).all() and (one["cols"] == many["cols"]).all()
    assert many["stats"]["split_k"] == split
    assert rel_fro(many["data"], one["data"]) <= 1e-14
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, 0.0, "T", "N")
    assert rel_fro(many["data"], ref["data"]) <= TOL_FP64


def test_split_k_with_cin_and_auto():
    p = _mixed(6, nb=(12, 400, 10), occ=0.2, alpha=0.75, beta=-1.25)
    check_parity(p, split_k=4)
    check_parity(p, split_k=0)


def test_deterministic_repeat():
    p = banded(seed=7, nb=200, eps=1e-8)
    a = run_multiply(p, stacks=False)
    b = run_multiply(p, stacks=False)
    assert (a["data"] == b["data"]).all()
    c = run_multiply(p, split_k=4, stacks=False)
    d = run_multiply(p, split_k=4, stacks=False)
    assert (c["data"] == d["data"]).all()


def test_beta_zero_ignores_nan_cin():
    p = _mixed(8, beta=0.0)
    p.C_in.data[:] = np.nan
    got, _ = check_parity(p)
    assert np.isfinite(got["data"]).all()


def test_empty_operands():
    rng = np.random.default_rng(9)
    s = np.full(6, 5, np.int32)
    A = BSMatrix(s, s, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = random_matrix(rng, s, s, 0.5)
    got, ref = check_parity(Problem(A, B))
    assert len(got["rows"]) == 0
    # empty product but C_in present: C_out = beta * C_in
    Ci = random_matrix(rng, s, s, 0.5)
    check_parity(Problem(A, B, Ci, 1.0, 3.0))


def test_filter_drops_everything():
    p = _mixed(10, eps=1e30, cin=False)
    got, ref = check_parity(p)
    assert got["stats"]["n_stack"] == 0 and len(got["rows"]) == 0


def test_error_codes_through_abi():
    ctx = bst.context()
    with pytest.raises(bst.BstError) as e:
        bst.bst_matrix_create(ctx, [5, 5], [5], [0, 0], [0, 0])
    assert e.value.name == "BST_ERR_DUPLICATE_BLOCK"
    with pytest.raises(bst.BstError) as e:
        bst.bst_matrix_create(ctx, [5, 5], [5], [2], [0])
    assert e.value.name == "BST_ERR_OUT_OF_RANGE"
    with pytest.raises(bst.BstError) as e:
        bst.bst_matrix_create(ctx, [5, 0], [5], [0], [0])
    assert e.value.name == "BST_ERR_INVALID_ARG"
    p = _mixed(11)
    from gpu_util import to_lib
    A, B = to_lib(p.A), to_lib(p.B)
    with pytest.raises(bst.BstError) as e:
        bst.multiply_plan(B, B)  # inner sizes differ
    assert e.value.name == "BST_ERR_SHAPE_MISMATCH"
    with pytest.raises(bst.BstError) as e:
        bst.multiply_plan(A, B, eps=-1.0)
    assert e.value.name == "BST_ERR_INVALID_ARG"
    plan = bst.multiply_plan(A, B)
    with pytest.raises(bst.BstError) as e:
        plan.execute()  # C_out data not bound
    assert e.value.name == "BST_ERR_STATE"


def test_banded_full_size_sampled():
    """The 4000x4000-block banded workload at full size: stack counts against the
    closed form of the candidate count, and 64 sampled C blocks against the oracle."""
    p = banded()
    got = run_multiply(p, stacks=False)
    st = got["stats"]
    rng = np.random.default_rng(0)
    sel = rng.choice(len(got["rows"]), 64, replace=False)
    bi, bj = got["rows"][sel], got["cols"][sel]
    vals, present = oracle.multiply_sample(p.A, p.B, None, 1.0, 0.0, p.eps, bi, bj,
                                           row_sizes=p.A.row_sizes, col_sizes=p.B.col_sizes)
    assert present.all()
    gv = np.concatenate([got["data"][got["offsets"][s]:got["offsets"][s] +
                                     p.A.row_sizes[got["rows"][s]] * p.B.col_sizes[got["cols"][s]]]
                         for s in sel])
    assert rel_fro(gv, vals) <= TOL_FP64
    # candidate count = sum_k nnzcol_A(k) nnzrow_B(k)
    ca = np.bincount(p.A.cols, minlength=len(p.A.col_sizes))
    rb = np.bincount(p.B.rows, minlength=len(p.B.row_sizes))
    assert st["n_candidates"] == int((ca.astype(np.int64) * rb).sum())
    assert 0 < st["n_filtered"] < st["n_candidates"]
