"""The block post-filter (bst_matrix_filter) and the chained filtered products of the
matrix-sign iteration on the GPU, against the CPU oracle: kept patterns and copied data
bit-exact, iterates within 1e-12 relative Frobenius error."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from paper_1910_13555_gb300 import bst, sign
from paper_1910_13555_gb300.workloads import banded, sign_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _host(m):
    rows, cols, _ = m.index()
    n = m.info[3]
    return rows, cols, m.data[:n].cpu().numpy()


def _gap_eps(norms, q):
    """An eps between two sorted norms that differ by > 1 %, near quantile q (no norm is
    within rounding of it, so both sides take the same decisions)."""
    s = np.sort(norms)
    i = int(q * len(s))
    while i + 1 < len(s) and s[i + 1] < 1.01 * s[i]:
        i += 1
    return float(np.sqrt(s[i] * s[i + 1]))


@pytest.mark.parametrize("q", [0.0, 0.3, 0.8])
def test_filter_matches_oracle(q):
    p = banded(seed=31, nb=300, decay=40.0, value_decay=8.0)
    norms = oracle.block_norms(p.A)
    eps = 0.0 if q == 0.0 else _gap_eps(norms, q)
    ref = oracle.filter_blocks(p.A, eps)
    X = to_lib(p.A)
    Y = bst.filter_blocks(X, eps)
    rows, cols, data = _host(Y)
    assert (rows == ref.rows).all() and (cols == ref.cols).all()
    assert (data == ref.data).all()


def test_filter_of_a_product_and_errors():
    import torch
    p = banded(seed=32, nb=200, decay=30.0, value_decay=8.0)
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply(A, B, None, 1.0, 0.0, p.eps)
    torch.cuda.synchronize()
    r = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    C_ref = oracle._Blocks(p.A.row_sizes, p.B.col_sizes, r["rows"], r["cols"], r["data"])
    eps = _gap_eps(oracle.block_norms(C_ref), 0.5)
    ref = oracle.filter_blocks(C_ref, eps)
    Y = bst.filter_blocks(plan.result, eps)
    rows, cols, data = _host(Y)
    assert (rows == ref.rows).all() and (cols == ref.cols).all()
    assert rel_fro(data, ref.data) <= 1e-12
    # a filter result belongs to its source: copying from another matrix is refused
    with pytest.raises(bst.BstError) as e:
        bst.bst_matrix_filter_copy(A.handle, Y.handle)
    assert e.value.name == "BST_ERR_SHAPE_MISMATCH"
    with pytest.raises(bst.BstError) as e:
        bst.bst_matrix_filter(bst.context(), A.handle, -1.0)
    assert e.value.name == "BST_ERR_INVALID_ARG"


def test_sign_iteration_matches_oracle():
    m = sign_matrix(seed=33, nb=80, width=3, p=0.6)
    X = to_lib(m)
    xs, stats = sign.sign_iteration(X, 4)
    ref = oracle.sign_iteration(m, 4)
    for x, r in zip(xs, ref):
        rows, cols, data = _host(x)
        assert (rows == r.rows).all() and (cols == r.cols).all()
        assert rel_fro(data, r.data) <= 1e-12
    assert all(s["flops"] > 0 for s in stats)


def test_sign_iteration_with_post_filter_converges():
    from helpers import densify
    from paper_1910_13555_gb300.workloads import BSMatrix
    m = sign_matrix(seed=34, nb=60, width=3, p=0.6)
    X = to_lib(m)
    full, _ = sign.sign_iteration(X, 12)
    filt, st = sign.sign_iteration(X, 12, eps_post=1e-9)
    assert st[-1]["blocks_X"] <= full[-1].info[2]

    def dense(x):
        rows, cols, data = _host(x)
        return densify(BSMatrix(m.row_sizes, m.col_sizes, rows, cols, data))

    F = dense(filt[-1])
    n = F.shape[0]
    # X converges to sign(H): X^2 = I
    assert np.linalg.norm(F @ F - np.eye(n)) <= 1e-6 * np.sqrt(n)
    assert np.linalg.norm(F - dense(full[-1])) <= 1e-6 * np.linalg.norm(F)
