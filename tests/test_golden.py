"""The golden fixtures of tests/golden/ (integer-valued problems, results exact in FP64):
the oracle still reproduces every stored value bit for bit, and the stored results
equal independent brute force on the same inputs -- a Python block loop with numpy
norms and products for the multiply (paper Sec. 2, Sec. 3.1), a pair loop of
np.einsum over the kept tensor-block pairs for the contraction (Sec. 4) -- also bit
for bit, because every partial sum is an integer."""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from helpers import brute_multiply, einsum_spec, tensor_dense
from paper_1910_13555_gb300.workloads import BSMatrix, BSTensor

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(glob.glob(os.path.join(GOLDEN, "*.json")))


def load(path):
    with open(path) as f:
        return json.load(f)


def mat(d):
    if d is None:
        return None
    return BSMatrix(np.asarray(d["row_sizes"], np.int32), np.asarray(d["col_sizes"], np.int32),
                    np.asarray(d["rows"], np.int32), np.asarray(d["cols"], np.int32),
                    np.asarray(d["data"], np.float64))


def ten(d):
    bs = [np.asarray(s, np.int32) for s in d["block_sizes"]]
    return BSTensor(bs, np.asarray(d["index"], np.int32).reshape(-1, len(bs)),
                    np.asarray(d["data"], np.float64))


def test_fixtures_present():
    names = {os.path.basename(f) for f in FILES}
    assert {"multiply_int_filter.json", "multiply_int_trans.json",
            "contract_int_rank4.json"} <= names


@pytest.mark.parametrize("path", FILES, ids=os.path.basename)
def test_oracle_reproduces_fixture(path):
    g = load(path)
    e = g["expected"]
    if g["op"] == "multiply":
        r = oracle.multiply(mat(g["A"]), mat(g["B"]), mat(g["C_in"]), g["alpha"], g["beta"],
                            g["eps"], g["transa"], g["transb"])
        for k in ("rows", "cols", "offsets", "mnk", "bucket_ptr", "a_off", "b_off", "c_off"):
            assert np.array_equal(np.asarray(r[k]).ravel(), np.asarray(e[k]).ravel()), k
        assert r["nfiltered"] == e["nfiltered"]
    else:
        r = oracle.contract(ten(g["T1"]), ten(g["T2"]), g["c1"], g["c2"], g["f1"], g["f2"],
                            g["result_order"], ten(g["R_in"]), g["alpha"], g["beta"], g["eps"])
        assert np.array_equal(r["index"].ravel(), np.asarray(e["index"]).ravel())
        assert np.array_equal(r["offsets"], np.asarray(e["offsets"]))
        assert (r["npairs"], r["nfiltered"]) == (e["npairs"], e["nfiltered"])
    assert np.array_equal(r["data"], np.asarray(e["data"], np.float64))


def _stacks_brute(A, B, kept, rows_c, cols_c, offs_c, transa, transb):
    """(m,n,k) buckets and (a_off, b_off, c_off) of the kept products, sorted by the
    bucket sizes then (i, j, k), rebuilt from the block index alone."""
    def where(M, tr):
        d = {}
        for b, o in enumerate(M.offsets):
            i, j = int(M.rows[b]), int(M.cols[b])
            d[(i, j) if tr == "N" else (j, i)] = int(o)
        return d
    ao, bo = where(A, transa), where(B, transb)
    co = {(int(i), int(j)): int(o) for i, j, o in zip(rows_c, cols_c, offs_c)}
    rs = A.row_sizes if transa == "N" else A.col_sizes
    ks = A.col_sizes if transa == "N" else A.row_sizes
    cs = B.col_sizes if transb == "N" else B.row_sizes
    ent = sorted((int(rs[i]), int(cs[j]), int(ks[k]), i, j, k) for i, j, k in kept)
    return ([(m, n, k) for m, n, k, *_ in ent], [ao[(i, k)] for *_, i, j, k in ent],
            [bo[(k, j)] for *_, i, j, k in ent], [co[(i, j)] for *_, i, j, k in ent])


@pytest.mark.parametrize("name", ["multiply_int_filter.json", "multiply_int_trans.json"])
def test_multiply_fixture_vs_block_loop(name):
    g = load(os.path.join(GOLDEN, name))
    e = g["expected"]
    A, B, Ci = mat(g["A"]), mat(g["B"]), mat(g["C_in"])
    blocks, kept, nfilt = brute_multiply(A, B, Ci, g["alpha"], g["beta"], g["eps"],
                                         g["transa"], g["transb"])
    assert nfilt == e["nfiltered"]
    keys = sorted(blocks)
    assert [k[0] for k in keys] == e["rows"] and [k[1] for k in keys] == e["cols"]
    data = np.concatenate([blocks[k].ravel() for k in keys])
    assert np.array_equal(data, np.asarray(e["data"], np.float64))
    mnk, a_off, b_off, c_off = _stacks_brute(A, B, kept, e["rows"], e["cols"], e["offsets"],
                                             g["transa"], g["transb"])
    bp = np.asarray(e["bucket_ptr"])
    emnk = np.asarray(e["mnk"]).reshape(-1, 3)
    assert [tuple(emnk[b]) for b in range(len(emnk)) for _ in range(bp[b], bp[b + 1])] == mnk
    assert (e["a_off"], e["b_off"], e["c_off"]) == (a_off, b_off, c_off)


def test_contract_fixture_vs_pair_loop():
    g = load(os.path.join(GOLDEN, "contract_int_rank4.json"))
    e = g["expected"]
    T1, T2, Rin = ten(g["T1"]), ten(g["T2"]), ten(g["R_in"])
    c1, c2, f1, f2, ro = g["c1"], g["c2"], g["f1"], g["f2"], g["result_order"]
    spec = einsum_spec(T1.rank, T2.rank, c1, c2, f1, f2, ro)
    o1, o2, l1, l2 = T1.offsets, T2.offsets, T1.block_lens, T2.block_lens
    acc = 0.0
    npairs = nfilt = 0
    kept_out = set()
    for a in range(T1.nblocks):
        for b in range(T2.nblocks):
            if any(T1.index[a][x] != T2.index[b][y] for x, y in zip(c1, c2)):
                continue
            x1, x2 = T1.data[o1[a]:o1[a] + l1[a]], T2.data[o2[b]:o2[b] + l2[b]]
            if np.linalg.norm(x1) * np.linalg.norm(x2) < g["eps"]:
                nfilt += 1
                continue
            npairs += 1
            t1 = BSTensor(T1.block_sizes, T1.index[a:a + 1], x1)
            t2 = BSTensor(T2.block_sizes, T2.index[b:b + 1], x2)
            acc = acc + np.einsum(spec, tensor_dense(t1), tensor_dense(t2))
            free = [T1.index[a][d] for d in f1] + [T2.index[b][d] for d in f2]
            kept_out.add(tuple(int(free[r]) for r in ro))
    assert (npairs, nfilt) == (e["npairs"], e["nfiltered"])
    pattern = sorted(kept_out | {tuple(int(v) for v in t) for t in Rin.index})
    assert [tuple(t) for t in e["index"]] == pattern
    rsizes = [([T1.block_sizes[d] for d in f1] + [T2.block_sizes[d] for d in f2])[r] for r in ro]
    R = BSTensor(rsizes, np.asarray(e["index"], np.int32), np.asarray(e["data"], np.float64))
    want = g["alpha"] * acc + g["beta"] * tensor_dense(Rin)
    assert np.array_equal(tensor_dense(R), want)
