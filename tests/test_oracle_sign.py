"""Pins of the oracle's block post-filter and of the chained sign iteration (paper Sec. 2:
chains of filtered products) against what the mathematics fixes: the filter keeps
exactly the blocks of norm >= eps with their data untouched (checked against norms
computed here from the densified blocks); on a block-diagonal matrix of scaled identity
blocks the iteration reduces to the scalar recurrence x <- (3x - x^3)/2; on a small
symmetric matrix it converges to sign(H) from an eigendecomposition."""
import numpy as np

import oracle
from helpers import block_of, densify
from paper_1910_13555_gb300.workloads import BSMatrix, sign_matrix


def _mat_from_blocks(sizes, blocks):
    keys = sorted(blocks)
    rows = np.array([k[0] for k in keys], np.int32)
    cols = np.array([k[1] for k in keys], np.int32)
    data = np.concatenate([np.asarray(blocks[k], np.float64).ravel() for k in keys])
    sz = np.asarray(sizes, np.int32)
    return BSMatrix(sz, sz, rows, cols, data)


def test_filter_keeps_exactly_the_blocks_above_eps():
    rng = np.random.default_rng(0)
    sizes = [2, 3, 5, 3]
    blocks = {}
    for i in range(4):
        for j in range(4):
            if rng.random() < 0.7:
                blocks[(i, j)] = rng.standard_normal((sizes[i], sizes[j])) * 10.0 ** -rng.uniform(0, 4)
    m = _mat_from_blocks(sizes, blocks)
    norms = np.array([np.sqrt(np.sum(block_of(m, b) ** 2)) for b in range(m.nblocks)])
    eps = float(np.median(norms)) * 1.0001
    f = oracle.filter_blocks(m, eps)
    keep = norms >= eps
    assert (f.rows == m.rows[keep]).all() and (f.cols == m.cols[keep]).all()
    kept = np.concatenate([block_of(m, b).ravel() for b in range(m.nblocks) if keep[b]])
    assert (f.data == kept).all()
    # eps = 0 keeps everything (zero blocks included), eps above every norm keeps nothing
    m.data[:m.block_lens[0]] = 0.0
    assert oracle.filter_blocks(m, 0.0).nblocks == m.nblocks
    assert oracle.filter_blocks(m, 1.0 + norms.max()).nblocks == 0


def test_filter_norm_of_identity_block():
    m = _mat_from_blocks([4, 9], {(0, 0): np.eye(4), (1, 1): np.eye(9)})
    # ||I_n||_F = sqrt(n): 2 and 3
    assert oracle.filter_blocks(m, 2.0).nblocks == 2
    assert oracle.filter_blocks(m, 2.5).nblocks == 1
    assert oracle.filter_blocks(m, 3.0).nblocks == 1
    assert oracle.filter_blocks(m, 3.0000001).nblocks == 0


def test_sign_iteration_scalar_recurrence():
    """Block-diagonal a_i I blocks: every iterate is diag(x_i(k)) with x <- (3x - x^3)/2."""
    sizes = [2, 5, 3]
    a = [0.3, -0.7, 0.9]
    m = _mat_from_blocks(sizes, {(i, i): a[i] * np.eye(sizes[i]) for i in range(3)})
    xs = oracle.sign_iteration(m, 6)
    x = np.array(a)
    for it in xs:
        x = (3.0 * x - x ** 3) / 2.0
        d = densify(BSMatrix(np.asarray(sizes, np.int32), np.asarray(sizes, np.int32), it.rows,
                             it.cols, it.data))
        want = np.diag(np.repeat(x, sizes))
        np.testing.assert_allclose(d, want, rtol=0, atol=1e-15)
        assert it.nblocks == 3


def test_sign_iteration_converges_to_sign_of_h():
    m = sign_matrix(seed=3, nb=12, width=2, p=0.8, sizes=(np.array([2, 3]), np.array([0.5, 0.5])))
    H = densify(m)
    np.testing.assert_allclose(H, H.T, atol=1e-15)
    w, v = np.linalg.eigh(H)
    assert np.abs(w).min() > 0.05 and np.abs(w).max() <= 1.0 + 1e-12
    S = (v * np.sign(w)) @ v.T
    xs = oracle.sign_iteration(m, 25)
    last = densify(BSMatrix(m.row_sizes, m.col_sizes, xs[-1].rows, xs[-1].cols, xs[-1].data))
    np.testing.assert_allclose(last, S, atol=1e-10)
    # the chain keeps X symmetric and every iterate commutes with H
    np.testing.assert_allclose(last, last.T, atol=1e-12)


def test_sign_iteration_post_filter_drops_blocks():
    m = sign_matrix(seed=4, nb=30, width=3, p=0.7, coupling=0.05)
    full = oracle.sign_iteration(m, 3)
    filt = oracle.sign_iteration(m, 3, eps_post=1e-4)
    assert filt[-1].nblocks < full[-1].nblocks
    # the dropped mass is small: the filtered iterate stays close
    a = densify(BSMatrix(m.row_sizes, m.col_sizes, full[-1].rows, full[-1].cols, full[-1].data))
    b = densify(BSMatrix(m.row_sizes, m.col_sizes, filt[-1].rows, filt[-1].cols, filt[-1].data))
    assert np.linalg.norm(a - b) < 1e-2 * np.linalg.norm(a)
