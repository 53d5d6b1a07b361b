"""Pins of the CPU oracle's block-sparse tensor contraction (paper Sec. 4) against
np.einsum on densified tensors, a brute-force block-pair loop for the filter, the
matrix special case, and the adjoint (dense einsum masked to the input patterns,
dot-product identity, central differences)."""
import numpy as np
import pytest

import oracle
from helpers import (einsum_spec, tensor_block_mask, tensor_dense, tensor_from_result)
from paper_1910_13555_gb300.workloads import BSTensor, random_tensor, rank3

SZ = np.array([2, 3, 5], np.int32)


def _sizes(rng, n):
    return rng.choice(SZ, n).astype(np.int32)


CASES = [
    # (rank1, rank2, c1, c2, f1, f2, result_order)
    (3, 3, [2], [0], [0, 1], [1, 2], None),
    (3, 3, [0, 2], [0, 1], [1], [2], None),            # the rank-3 workload's pattern
    (3, 3, [0, 2], [0, 1], [1], [2], [1, 0]),
    (4, 3, [1, 3], [2, 0], [0, 2], [1], [2, 0, 1]),
    (4, 4, [0, 1, 2], [3, 1, 0], [3], [2], [1, 0]),
    (2, 2, [0], [0], [1], [1], None),                  # A^T B
    (4, 2, [3], [0], [0, 1, 2], [1], [3, 1, 0, 2]),
]


def _make(seed, case, occ=0.5):
    r1, r2, c1, c2, f1, f2, ro = case
    rng = np.random.default_rng(seed)
    nb1 = [int(rng.integers(2, 4)) for _ in range(r1)]
    s1 = [_sizes(rng, n) for n in nb1]
    nb2 = [0] * r2
    s2 = [None] * r2
    for a, b in zip(c1, c2):
        nb2[b] = nb1[a]
        s2[b] = s1[a]
    for b in f2:
        nb2[b] = int(rng.integers(2, 4))
        s2[b] = _sizes(rng, nb2[b])
    T1 = random_tensor(rng, nb1, s1, occ)
    T2 = random_tensor(rng, nb2, s2, occ)
    return T1, T2


def _result_sizes(T1, T2, case):
    _, _, c1, c2, f1, f2, ro = case
    free = [T1.block_sizes[a] for a in f1] + [T2.block_sizes[b] for b in f2]
    ro = ro if ro is not None else list(range(len(free)))
    return [free[r] for r in ro]


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_contract_vs_einsum(seed, ci):
    case = CASES[ci]
    r1, r2, c1, c2, f1, f2, ro = case
    T1, T2 = _make(seed * 10 + ci, case)
    rs = _result_sizes(T1, T2, case)
    rng = np.random.default_rng(seed)
    Rin = random_tensor(rng, [len(s) for s in rs], rs, 0.4)
    alpha, beta = 0.75, -1.5
    res = oracle.contract(T1, T2, c1, c2, f1, f2, ro, Rin, alpha, beta, 0.0)
    R = tensor_from_result(res, rs)
    spec = einsum_spec(r1, r2, c1, c2, f1, f2, ro)
    ref = alpha * np.einsum(spec, tensor_dense(T1), tensor_dense(T2)) + beta * tensor_dense(Rin)
    np.testing.assert_allclose(tensor_dense(R), ref, rtol=0,
                               atol=1e-13 * max(1.0, np.abs(ref).max()))
    # the result pattern: every block tuple reachable by some block pair, plus R_in's
    expect = set(map(tuple, Rin.index.tolist()))
    for b1 in T1.index.tolist():
        for b2 in T2.index.tolist():
            if all(b1[a] == b2[b] for a, b in zip(c1, c2)):
                free = [b1[a] for a in f1] + [b2[b] for b in f2]
                order = ro if ro is not None else range(len(free))
                expect.add(tuple(free[r] for r in order))
    assert set(map(tuple, res["index"].tolist())) == expect
    assert res["index"].tolist() == sorted(res["index"].tolist())


def test_contract_filter_vs_pair_loop():
    case = CASES[1]
    r1, r2, c1, c2, f1, f2, ro = case
    T1, T2 = _make(77, case, occ=0.7)
    rng = np.random.default_rng(5)
    T1.data *= np.repeat(10.0 ** -rng.uniform(0, 3, T1.nblocks), T1.block_lens)
    offs1, offs2 = T1.offsets, T2.offsets
    n1 = np.array([np.linalg.norm(T1.data[offs1[b]:offs1[b] + T1.block_lens[b]])
                   for b in range(T1.nblocks)])
    n2 = np.array([np.linalg.norm(T2.data[offs2[b]:offs2[b] + T2.block_lens[b]])
                   for b in range(T2.nblocks)])
    pairs = [(a, b) for a in range(T1.nblocks) for b in range(T2.nblocks)
             if all(T1.index[a][x] == T2.index[b][y] for x, y in zip(c1, c2))]
    pn = sorted(n1[a] * n2[b] for a, b in pairs)
    eps = float(np.sqrt(pn[len(pn) // 2] * pn[len(pn) // 2 + 1]))
    res = oracle.contract(T1, T2, c1, c2, f1, f2, ro, None, 1.0, 0.0, eps)
    kept = [(a, b) for a, b in pairs if n1[a] * n2[b] >= eps]
    assert res["npairs"] == len(kept) and res["nfiltered"] == len(pairs) - len(kept)
    # dense reference from the kept pairs only: mask T1/T2 per pair
    spec = einsum_spec(r1, r2, c1, c2, f1, f2, ro)
    rs = _result_sizes(T1, T2, case)
    acc = 0.0
    for a, b in kept:
        t1 = BSTensor(T1.block_sizes, T1.index[a:a + 1],
                      T1.data[offs1[a]:offs1[a] + T1.block_lens[a]])
        t2 = BSTensor(T2.block_sizes, T2.index[b:b + 1],
                      T2.data[offs2[b]:offs2[b] + T2.block_lens[b]])
        acc = acc + np.einsum(spec, tensor_dense(t1), tensor_dense(t2))
    np.testing.assert_allclose(tensor_dense(tensor_from_result(res, rs)), acc, rtol=0,
                               atol=1e-13 * np.abs(acc).max())


def test_contract_matrix_case_equals_transposed_multiply():
    """A rank-2 contraction over mode 0 of both is A^T B (paper Sec. 3.1)."""
    from paper_1910_13555_gb300.workloads import BSMatrix
    case = CASES[5]
    T1, T2 = _make(3, case)
    res = oracle.contract(T1, T2, [0], [0], [1], [1])
    A = BSMatrix(T1.block_sizes[0], T1.block_sizes[1], T1.index[:, 0], T1.index[:, 1], T1.data)
    B = BSMatrix(T2.block_sizes[0], T2.block_sizes[1], T2.index[:, 0], T2.index[:, 1], T2.data)
    m = oracle.multiply(A, B, None, 1.0, 0.0, 0.0, "T", "N")
    assert (res["index"][:, 0] == m["rows"]).all() and (res["index"][:, 1] == m["cols"]).all()
    np.testing.assert_allclose(res["data"], m["data"], rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("ci", [0, 1, 3, 4])
def test_contract_adjoint(ci):
    case = CASES[ci]
    r1, r2, c1, c2, f1, f2, ro = case
    T1, T2 = _make(500 + ci, case)
    alpha = 1.25
    res = oracle.contract(T1, T2, c1, c2, f1, f2, ro, None, alpha, 0.0, 0.0)
    rs = _result_sizes(T1, T2, case)
    rng = np.random.default_rng(ci)
    G = rng.standard_normal(len(res["data"]))
    d1, d2, _ = oracle.contract_adjoint(T1, T2, c1, c2, f1, f2, ro, None, alpha, 0.0, 0.0, G)
    Gd = tensor_dense(BSTensor(rs, res["index"], G))
    # dense adjoints by einsum with the roles permuted, masked to the input patterns
    spec = einsum_spec(r1, r2, c1, c2, f1, f2, ro)
    ins, out = spec.split("->")
    s1, s2 = ins.split(",")
    g1 = alpha * np.einsum(f"{out},{s2}->{s1}", Gd, tensor_dense(T2))
    g2 = alpha * np.einsum(f"{s1},{out}->{s2}", tensor_dense(T1), Gd)
    D1 = tensor_dense(BSTensor(T1.block_sizes, T1.index, d1))
    D2 = tensor_dense(BSTensor(T2.block_sizes, T2.index, d2))
    np.testing.assert_allclose(D1, np.where(tensor_block_mask(T1), g1, 0.0), atol=1e-12)
    np.testing.assert_allclose(D2, np.where(tensor_block_mask(T2), g2, 0.0), atol=1e-12)
    lhs = np.dot(G, res["data"])
    np.testing.assert_allclose(np.dot(d1, T1.data), lhs, rtol=1e-12)
    np.testing.assert_allclose(np.dot(d2, T2.data), lhs, rtol=1e-12)


def test_contract_adjoint_finite_difference_rank3():
    w = rank3(seed=9, nP=6, sP=3, nao=8, window=4, p=0.6)
    T, U = w.T1, w.T2
    args = (w.c1, w.c2, w.f1, w.f2, w.result_order, None, 1.0, 0.0, 0.0)
    res = oracle.contract(T, U, *args[:5], None, 1.0, 0.0, 0.0)
    dT, dU, _ = oracle.contract_adjoint(T, U, *args, res["data"])
    L = 0.5 * np.sum(res["data"] ** 2)
    rng = np.random.default_rng(2)
    h = 1e-6
    for M, g in ((T, dT), (U, dU)):
        for e in rng.choice(len(M.data), 10, replace=False):
            old = M.data[e]
            M.data[e] = old + h
            lp = 0.5 * np.sum(oracle.contract(T, U, *args[:5], None, 1.0, 0.0, 0.0)["data"] ** 2)
            M.data[e] = old - h
            lm = 0.5 * np.sum(oracle.contract(T, U, *args[:5], None, 1.0, 0.0, 0.0)["data"] ** 2)
            M.data[e] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[e]) <= 1e-7 * max(1, abs(g[e])) + 8 * 2.0 ** -52 * L / h


def test_contract_errors():
    case = CASES[0]
    T1, T2 = _make(1, case)
    with pytest.raises(oracle.OracleError) as e:
        oracle.contract(T1, T2, [2], [1], [0, 1], [0, 2])   # mismatched contracted sizes
    assert e.value.name in ("SHAPE_MISMATCH", "INVALID_ARG")
    with pytest.raises(oracle.OracleError) as e:
        oracle.contract(T1, T2, [2, 2], [0, 1], [0], [2])   # mode listed twice
    assert e.value.name == "INVALID_ARG"


def test_contract_sample_matches_full():
    case = CASES[3]
    r1, r2, c1, c2, f1, f2, ro = case
    T1, T2 = _make(42, case)
    rs = _result_sizes(T1, T2, case)
    Rin = random_tensor(np.random.default_rng(3), [len(s) for s in rs], rs, 0.4)
    full = oracle.contract(T1, T2, c1, c2, f1, f2, ro, Rin, 0.5, 2.0, 0.0)
    sel = np.arange(0, len(full["index"]), 3)
    vals, present = oracle.contract_sample(T1, T2, c1, c2, f1, f2, ro, Rin, 0.5, 2.0, 0.0,
                                           full["index"][sel], rs)
    assert present.all()
    lens = np.ones(len(full["index"]), np.int64)
    for d, sz in enumerate(rs):
        lens *= np.asarray(sz, np.int64)[full["index"][:, d]]
    ref = np.concatenate([full["data"][full["offsets"][b]:full["offsets"][b] + lens[b]] for b in sel])
    np.testing.assert_allclose(vals, ref, rtol=1e-14, atol=1e-14)
