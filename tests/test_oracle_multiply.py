"""Pins of the CPU oracle's block-sparse multiply against things other than itself:
dense brute force (numpy @), a Python block loop with numpy norms, closed forms
(identity blocks, all-present blocks == textbook GEMM), counting formulas and
invariants (associativity over the pattern, filter monotonicity, transpose identity).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from helpers import (block_of, brute_multiply, densify, from_result, pattern_dense,
                     random_matrix, transpose_matrix)
from paper_1910_13555_gb300.workloads import BSMatrix, plain, banded, tall_skinny

SZ = np.array([5, 13, 23, 1, 7], np.int32)


def _case(seed, nb_m=6, nb_k=7, nb_n=5, occ=0.35, mixed=True):
    rng = np.random.default_rng(seed)
    pick = (lambda n: rng.choice(SZ, n).astype(np.int32)) if mixed else (
        lambda n: np.full(n, 5, np.int32))
    m, k, n = pick(nb_m), pick(nb_k), pick(nb_n)
    A = random_matrix(rng, m, k, occ)
    B = random_matrix(rng, k, n, occ)
    Ci = random_matrix(rng, m, n, occ * 0.5)
    return A, B, Ci


def _dense_result(res, row_sizes, col_sizes):
    return densify(from_result(res, row_sizes, col_sizes))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_multiply_vs_dense(seed, ta, tb):
    A, B, Ci = _case(seed)
    if ta == "T":
        A = transpose_matrix(A)
    if tb == "T":
        B = transpose_matrix(B)
    alpha, beta = 1.5, -0.75
    res = oracle.multiply(A, B, Ci, alpha, beta, 0.0, ta, tb)
    dA = densify(A).T if ta == "T" else densify(A)
    dB = densify(B).T if tb == "T" else densify(B)
    ref = alpha * dA @ dB + beta * densify(Ci)
    got = _dense_result(res, Ci.row_sizes, Ci.col_sizes)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))
    # pattern = boolean product of the patterns united with pattern(C_in)
    PA = pattern_dense(len(A.row_sizes), len(A.col_sizes), A.rows, A.cols)
    PB = pattern_dense(len(B.row_sizes), len(B.col_sizes), B.rows, B.cols)
    PA = PA.T if ta == "T" else PA
    PB = PB.T if tb == "T" else PB
    PC = (sp.csr_matrix(PA.astype(np.int64)) @ sp.csr_matrix(PB.astype(np.int64))).toarray() > 0
    PC |= pattern_dense(len(Ci.row_sizes), len(Ci.col_sizes), Ci.rows, Ci.cols)
    got_p = pattern_dense(*PC.shape, res["rows"], res["cols"])
    assert (got_p == PC).all()
    # stack count = sum_k nnzcol_opA(k) * nnzrow_opB(k)
    assert len(res["a_off"]) == int((PA.sum(0) * PB.sum(1)).sum())


@pytest.mark.parametrize("seed", range(4))
def test_multiply_filter_vs_block_loop(seed):
    rng = np.random.default_rng(100 + seed)
    A, B, Ci = _case(100 + seed, occ=0.5)
    # spread the block norms over decades so that the filter bites
    A.data *= np.repeat(10.0 ** -rng.uniform(0, 4, A.nblocks), A.block_lens)
    B.data *= np.repeat(10.0 ** -rng.uniform(0, 4, B.nblocks), B.block_lens)
    na = np.array([np.linalg.norm(block_of(A, b)) for b in range(A.nblocks)])
    nb = np.array([np.linalg.norm(block_of(B, b)) for b in range(B.nblocks)])
    prods = np.sort((na[:, None] * nb[None, :]).ravel())
    eps = float(np.sqrt(prods[len(prods) // 3] * prods[len(prods) // 3 + 1]))  # between two
    res = oracle.multiply(A, B, Ci, 2.0, 0.5, eps)
    ref, kept, nfilt = brute_multiply(A, B, Ci, 2.0, 0.5, eps)
    assert res["nfiltered"] == nfilt and nfilt > 0
    keys = list(zip(res["rows"].tolist(), res["cols"].tolist()))
    assert set(keys) == set(ref.keys())
    scale = max(np.abs(v).max() for v in ref.values())
    for b, key in enumerate(keys):
        m, n = Ci.row_sizes[key[0]], Ci.col_sizes[key[1]]
        blk = res["data"][res["offsets"][b]:res["offsets"][b] + m * n].reshape(m, n)
        np.testing.assert_allclose(blk, ref[key], rtol=1e-13, atol=1e-14 * scale)
    assert len(res["a_off"]) == len(kept)


def _stack_triples(res, A, B, ta="N", tb="N"):
    """Recover (i, j, k) of every stack entry from its offsets."""
    aoff = {int(o): b for b, o in enumerate(A.offsets)}
    boff = {int(o): b for b, o in enumerate(B.offsets)}
    coff = {int(o): b for b, o in enumerate(res["offsets"])}
    out = []
    for e in range(len(res["a_off"])):
        a, b, c = aoff[int(res["a_off"][e])], boff[int(res["b_off"][e])], coff[int(res["c_off"][e])]
        i, k = (A.rows[a], A.cols[a]) if ta == "N" else (A.cols[a], A.rows[a])
        k2, j = (B.rows[b], B.cols[b]) if tb == "N" else (B.cols[b], B.rows[b])
        assert k == k2 and (res["rows"][c], res["cols"][c]) == (i, j)
        out.append((int(i), int(j), int(k)))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_stack_order_and_buckets(seed):
    A, B, Ci = _case(200 + seed, nb_m=8, nb_k=9, nb_n=7)
    res = oracle.multiply(A, B, None, 1.0, 0.0, 0.0)
    tri = _stack_triples(res, A, B)
    mnk, bp = res["mnk"], res["bucket_ptr"]
    assert bp[0] == 0 and bp[-1] == len(tri)
    keys = [tuple(x) for x in mnk.tolist()]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    for q in range(len(keys)):
        seg = tri[bp[q]:bp[q + 1]]
        assert len(seg) > 0 and seg == sorted(seg)
        for (i, j, k) in seg:
            assert (A.row_sizes[i], B.col_sizes[j], A.col_sizes[k]) == keys[q]
    _, kept, _ = brute_multiply(A, B, None, 1.0, 0.0, 0.0)
    assert set(tri) == kept and len(tri) == len(kept)
    assert res["flops"] == sum(2.0 * m * n * k * (bp[q + 1] - bp[q])
                               for q, (m, n, k) in enumerate(keys))


def test_identity_blocks_closed_form():
    """A = block-diagonal identity => C = B exactly (every product is 1*x + 0*y)."""
    rng = np.random.default_rng(7)
    sz = rng.choice(SZ, 9).astype(np.int32)
    I = BSMatrix(sz, sz, np.arange(9, dtype=np.int32), np.arange(9, dtype=np.int32),
                 np.concatenate([np.eye(s).ravel() for s in sz]))
    B = random_matrix(rng, sz, sz, 0.4)
    res = oracle.multiply(I, B)
    assert (res["rows"] == B.rows).all() and (res["cols"] == B.cols).all()
    assert (res["data"] == B.data).all()


def test_all_present_is_dense_gemm():
    """Every block present, eps = 0: the textbook dense GEMM (integer data -> exact)."""
    rng = np.random.default_rng(8)
    m, k, n = (rng.choice(SZ, c).astype(np.int32) for c in (4, 5, 3))
    def full(r, c):
        R, Cc = np.meshgrid(np.arange(len(r)), np.arange(len(c)), indexing="ij")
        rows, cols = R.ravel().astype(np.int32), Cc.ravel().astype(np.int32)
        lens = r[rows].astype(np.int64) * c[cols]
        return BSMatrix(r, c, rows, cols, rng.integers(-9, 10, int(lens.sum())).astype(float))
    A, B = full(m, k), full(k, n)
    res = oracle.multiply(A, B)
    assert (_dense_result(res, m, n) == densify(A) @ densify(B)).all()


def test_associativity_over_pattern():
    rng = np.random.default_rng(9)
    s = rng.choice(SZ, 6).astype(np.int32)
    A, B, C = (random_matrix(rng, s, s, 0.3) for _ in range(3))
    AB = from_result(oracle.multiply(A, B), s, s)
    BC = from_result(oracle.multiply(B, C), s, s)
    L = oracle.multiply(AB, C)
    R = oracle.multiply(A, BC)
    assert (L["rows"] == R["rows"]).all() and (L["cols"] == R["cols"]).all()
    np.testing.assert_allclose(L["data"], R["data"], rtol=0,
                               atol=1e-12 * np.abs(R["data"]).max())


def test_filter_monotonicity():
    p = banded(seed=11, nb=60, occ=0.2, decay=10.0, value_decay=3.0, eps=1e-3)
    A, B = p.A, p.B
    prev = None
    for eps in [0.0, 1e-6, 1e-3, 1e-1, 1.0]:
        res = oracle.multiply(A, B, None, 1.0, 0.0, eps)
        tri = set(_stack_triples(res, A, B))
        pat = set(zip(res["rows"].tolist(), res["cols"].tolist()))
        if prev is not None:
            assert tri <= prev[0] and pat <= prev[1]
        prev = (tri, pat)
    assert len(prev[0]) < len(set(_stack_triples(oracle.multiply(A, B), A, B)))


def test_transpose_identity():
    """(A B)^T == B^T A^T with the transposes taken by the op flags."""
    A, B, _ = _case(12)
    L = oracle.multiply(A, B)
    R = oracle.multiply(B, A, None, 1.0, 0.0, 0.0, "T", "T")
    Lt = transpose_matrix(from_result(L, A.row_sizes, B.col_sizes))
    assert (Lt.rows == R["rows"]).all() and (Lt.cols == R["cols"]).all()
    np.testing.assert_allclose(R["data"], Lt.data, rtol=1e-14, atol=1e-14)


def test_beta_zero_does_not_read_cin():
    A, B, Ci = _case(13)
    Ci.data[:] = np.nan
    res = oracle.multiply(A, B, Ci, 1.0, 0.0, 0.0)
    assert np.isfinite(res["data"]).all()
    pat = set(zip(res["rows"].tolist(), res["cols"].tolist()))
    assert set(zip(Ci.rows.tolist(), Ci.cols.tolist())) <= pat


def test_sample_matches_full():
    A, B, Ci = _case(14)
    res = oracle.multiply(A, B, Ci, 0.5, 2.0, 0.0)
    sel = np.arange(0, len(res["rows"]), 2)
    vals, present = oracle.multiply_sample(A, B, Ci, 0.5, 2.0, 0.0, res["rows"][sel],
                                           res["cols"][sel], row_sizes=Ci.row_sizes,
                                           col_sizes=Ci.col_sizes)
    assert present.all()
    ref = np.concatenate([res["data"][res["offsets"][b]:res["offsets"][b] +
                                      Ci.row_sizes[res["rows"][b]] * Ci.col_sizes[res["cols"][b]]]
                          for b in sel])
    np.testing.assert_allclose(vals, ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_sample_filter_vs_block_loop(seed, ta, tb):
    """The sampled multiply at eps > 0 against the Python block loop under the same
    filter, on every block of the C grid (present or not).  The sample is chosen so that
    the filter changes values: a dropped or inverted norm test fails it."""
    rng = np.random.default_rng(300 + seed)
    A, B, Ci = _case(300 + seed, occ=0.5)
    A.data *= np.repeat(10.0 ** -rng.uniform(0, 4, A.nblocks), A.block_lens)
    B.data *= np.repeat(10.0 ** -rng.uniform(0, 4, B.nblocks), B.block_lens)
    if ta == "T":
        A = transpose_matrix(A)
    if tb == "T":
        B = transpose_matrix(B)
    na = np.array([np.linalg.norm(block_of(A, b)) for b in range(A.nblocks)])
    nb = np.array([np.linalg.norm(block_of(B, b)) for b in range(B.nblocks)])
    prods = np.sort((na[:, None] * nb[None, :]).ravel())
    eps = float(np.sqrt(prods[len(prods) // 2] * prods[len(prods) // 2 + 1]))
    alpha, beta = -1.5, 0.25
    ref, kept, nfilt = brute_multiply(A, B, Ci, alpha, beta, eps, ta, tb)
    unf, _, _ = brute_multiply(A, B, Ci, alpha, beta, 0.0, ta, tb)
    assert nfilt > 0
    nbr, nbc = len(Ci.row_sizes), len(Ci.col_sizes)
    bi, bj = (x.ravel().astype(np.int32) for x in np.meshgrid(np.arange(nbr), np.arange(nbc),
                                                               indexing="ij"))
    vals, present = oracle.multiply_sample(A, B, Ci, alpha, beta, eps, bi, bj, ta, tb,
                                           row_sizes=Ci.row_sizes, col_sizes=Ci.col_sizes)
    pos, changed = 0, 0
    for e in range(len(bi)):
        key = (int(bi[e]), int(bj[e]))
        m, n = int(Ci.row_sizes[key[0]]), int(Ci.col_sizes[key[1]])
        got = vals[pos:pos + m * n].reshape(m, n)
        pos += m * n
        assert present[e] == (key in ref), key
        want = ref.get(key, np.zeros((m, n)))
        scale = max(1e-300, np.abs(want).max())
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14 * scale)
        if key in unf and np.abs(unf[key] - want).max() > 1e-6 * max(scale, np.abs(unf[key]).max()):
            changed += 1
    assert changed > 0  # some sampled block holds a filtered product of visible size


def test_errors():
    A, B, Ci = _case(15)
    dup = BSMatrix(A.row_sizes, A.col_sizes, np.r_[A.rows, A.rows[:1]], np.r_[A.cols, A.cols[:1]],
                   np.r_[A.data, A.data[:A.block_lens[0]]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.multiply(dup, B)
    assert e.value.name == "DUPLICATE_BLOCK"
    bad = BSMatrix(A.row_sizes, A.col_sizes, A.rows.copy(), A.cols.copy(), A.data)
    bad.cols[0] = len(A.col_sizes)
    with pytest.raises(oracle.OracleError) as e:
        oracle.multiply(bad, B)
    assert e.value.name == "OUT_OF_RANGE"
    with pytest.raises(oracle.OracleError) as e:
        oracle.multiply(B, B)
    assert e.value.name == "SHAPE_MISMATCH"


def test_block_norms():
    A, _, _ = _case(16)
    n = oracle.block_norms(A)
    ref = [np.linalg.norm(block_of(A, b)) for b in range(A.nblocks)]
    np.testing.assert_allclose(n, ref, rtol=1e-15)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N")])
def test_adjoint_vs_dense_and_dot_identity(seed, ta, tb):
    A, B, Ci = _case(300 + seed)
    if ta == "T":
        A = transpose_matrix(A)
    alpha, beta = 1.25, 0.5
    res = oracle.multiply(A, B, Ci, alpha, beta, 0.0, ta, tb)
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(len(res["data"]))
    dA, dB, dCi = oracle.multiply_adjoint(A, B, Ci, alpha, beta, 0.0, G, ta, tb)
    Gd = densify(from_result(dict(res, data=G), Ci.row_sizes, Ci.col_sizes))
    opA = densify(A).T if ta == "T" else densify(A)
    opB = densify(B)
    gA = alpha * Gd @ opB.T
    gA = gA.T if ta == "T" else gA
    gB = alpha * opA.T @ Gd
    mA = densify(BSMatrix(A.row_sizes, A.col_sizes, A.rows, A.cols, np.ones_like(A.data))) > 0
    mB = densify(BSMatrix(B.row_sizes, B.col_sizes, B.rows, B.cols, np.ones_like(B.data))) > 0
    dAd = densify(BSMatrix(A.row_sizes, A.col_sizes, A.rows, A.cols, dA))
    dBd = densify(BSMatrix(B.row_sizes, B.col_sizes, B.rows, B.cols, dB))
    np.testing.assert_allclose(dAd, np.where(mA, gA, 0.0), atol=1e-12)
    np.testing.assert_allclose(dBd, np.where(mB, gB, 0.0), atol=1e-12)
    # dot-product identity <G, alpha op(A) op(B)> = <dA, A> = <dB, B>
    lhs = alpha * np.sum(Gd * (opA @ opB))
    np.testing.assert_allclose(np.dot(dA, A.data), lhs, rtol=1e-12)
    np.testing.assert_allclose(np.dot(dB, B.data), lhs, rtol=1e-12)
    # dC_in = beta * G restricted to the C_in blocks
    Cid = densify(BSMatrix(Ci.row_sizes, Ci.col_sizes, Ci.rows, Ci.cols, dCi))
    mC = densify(BSMatrix(Ci.row_sizes, Ci.col_sizes, Ci.rows, Ci.cols,
                          np.ones_like(Ci.data))) > 0
    np.testing.assert_allclose(Cid, np.where(mC, beta * Gd, 0.0), atol=1e-14)


def test_adjoint_finite_difference():
    """L = 1/2 ||C||^2 is quadratic in each entry, so central differences are exact up
    to rounding; the gradient is the adjoint applied to dC = C."""
    A, B, _ = _case(400)
    res = oracle.multiply(A, B)
    dA, dB, _ = oracle.multiply_adjoint(A, B, None, 1.0, 0.0, 0.0, res["data"])
    rng = np.random.default_rng(1)
    h = 1e-6
    for which, M, g in (("A", A, dA), ("B", B, dB)):
        for e in rng.choice(len(M.data), 8, replace=False):
            old = M.data[e]
            M.data[e] = old + h
            lp = 0.5 * np.sum(oracle.multiply(A, B)["data"] ** 2)
            M.data[e] = old - h
            lm = 0.5 * np.sum(oracle.multiply(A, B)["data"] ** 2)
            M.data[e] = old
            fd = (lp - lm) / (2 * h)
            L = 0.5 * np.sum(res["data"] ** 2)
            assert abs(fd - g[e]) <= 1e-7 * max(1, abs(g[e])) + 8 * 2.0 ** -52 * L / h


def test_workload_generators_reproducible():
    p1, p2 = plain(seed=5), plain(seed=5)
    assert (p1.A.data == p2.A.data).all() and (p1.B.rows == p2.B.rows).all()
    t = tall_skinny(seed=3, nk=2000, nmn=40, window=8, p=0.25)
    assert t.transa == "T" and t.A.nblocks > 0
    b = banded(seed=4, nb=300, eps=1e-8)
    assert b.A.nblocks > 0


def test_birthday_occupancy_of_c():
    """iid Bernoulli patterns: E[occ(C)] = 1 - (1 - pA pB)^K per block (pattern pin)."""
    rng = np.random.default_rng(21)
    nb, p = 120, 0.05
    s = np.full(nb, 1, np.int32)
    A = random_matrix(rng, s, s, p)
    B = random_matrix(rng, s, s, p)
    res = oracle.multiply(A, B)
    occ = len(res["rows"]) / nb / nb
    pa, pb = A.nblocks / nb / nb, B.nblocks / nb / nb
    expect = 1 - (1 - pa * pb) ** nb
    assert abs(occ - expect) < 4 * np.sqrt(expect * (1 - expect) / nb / nb) + 0.01
