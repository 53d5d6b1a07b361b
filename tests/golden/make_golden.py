"""Write the golden fixtures of this folder: small seeded block-sparse problems with
integer-valued entries and their results, computed by the CPU oracle alone.

    python tests/golden/make_golden.py

Every input entry is an integer in [-3, 3] and alpha, beta are small integers, so every
partial sum of the products is an integer far below 2^53: the results are exact in FP64
whatever the order of summation, and any correct implementation of the definitions
reproduces the stored values bit for bit.  The filter thresholds are k + 0.5 for an
integer k; a product of block norms is sqrt(integer * integer), so no filter decision
can tie with the threshold.

Definitions followed (paper Sec. 2: blocked CSR matrices of small dense blocks, the
product as a sum of block products gathered into stacks; Sec. 3.1: the transposed
tall-and-skinny product C = A^T B; Sec. 4: a tensor contraction recast as a matrix
product over folded indices).  The block-norm filter, the stack order and the result
permutation follow the readings stated beside the oracle.

This script is the only writer of the fixtures; it calls nothing but ``oracle`` and
plain numpy for the seeded inputs.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

SIZES = np.array([1, 2, 3, 5], np.int32)


def int_matrix(rng, row_sizes, col_sizes, occ):
    keep = rng.random((len(row_sizes), len(col_sizes))) < occ
    rows, cols = np.nonzero(keep)
    n = int((row_sizes[rows].astype(np.int64) * col_sizes[cols]).sum())
    return dict(row_sizes=row_sizes.tolist(), col_sizes=col_sizes.tolist(),
                rows=rows.astype(np.int32).tolist(), cols=cols.astype(np.int32).tolist(),
                data=rng.integers(-3, 4, n).astype(float).tolist())


def int_tensor(rng, block_sizes, occ):
    grids = np.stack(np.meshgrid(*[np.arange(len(s)) for s in block_sizes], indexing="ij"), -1)
    tuples = grids.reshape(-1, len(block_sizes))
    index = tuples[rng.random(len(tuples)) < occ]
    lens = np.ones(len(index), np.int64)
    for d, s in enumerate(block_sizes):
        lens *= np.asarray(s, np.int64)[index[:, d]]
    return dict(block_sizes=[np.asarray(s).tolist() for s in block_sizes],
                index=index.astype(np.int32).tolist(),
                data=rng.integers(-3, 4, int(lens.sum())).astype(float).tolist())


class M:
    """Attribute view of a stored matrix, as the oracle takes it."""

    def __init__(self, d):
        self.row_sizes = np.asarray(d["row_sizes"], np.int32)
        self.col_sizes = np.asarray(d["col_sizes"], np.int32)
        self.rows = np.asarray(d["rows"], np.int32)
        self.cols = np.asarray(d["cols"], np.int32)
        self.data = np.asarray(d["data"], np.float64)


class T:
    """Attribute view of a stored tensor, as the oracle takes it."""

    def __init__(self, d):
        self.block_sizes = [np.asarray(s, np.int32) for s in d["block_sizes"]]
        self.index = np.asarray(d["index"], np.int32).reshape(-1, len(self.block_sizes))
        self.data = np.asarray(d["data"], np.float64)


def _ints(a):
    return np.asarray(a).tolist()


def multiply_case(name, seed, nbr, nk, nbc, transa, transb, alpha, beta, eps, cin_occ):
    rng = np.random.default_rng(seed)
    rs = rng.choice(SIZES, nbr).astype(np.int32)
    ks = rng.choice(SIZES, nk).astype(np.int32)
    cs = rng.choice(SIZES, nbc).astype(np.int32)
    A = int_matrix(rng, ks, rs, 0.5) if transa == "T" else int_matrix(rng, rs, ks, 0.5)
    B = int_matrix(rng, cs, ks, 0.5) if transb == "T" else int_matrix(rng, ks, cs, 0.5)
    Cin = int_matrix(rng, rs, cs, cin_occ) if cin_occ > 0 else None
    ref = oracle.multiply(M(A), M(B), M(Cin) if Cin else None, alpha, beta, eps, transa, transb)
    return dict(
        name=name,
        cites="Sec. 2 (blocked CSR, sum of small dense block products in stacks)"
              + ("; Sec. 3.1 (C = A^T B, S_C << S_A, S_B)" if transa == "T" else ""),
        op="multiply", transa=transa, transb=transb, alpha=alpha, beta=beta, eps=eps,
        A=A, B=B, C_in=Cin,
        expected=dict(rows=_ints(ref["rows"]), cols=_ints(ref["cols"]),
                      offsets=_ints(ref["offsets"]), data=_ints(ref["data"]),
                      mnk=_ints(ref["mnk"]), bucket_ptr=_ints(ref["bucket_ptr"]),
                      a_off=_ints(ref["a_off"]), b_off=_ints(ref["b_off"]),
                      c_off=_ints(ref["c_off"]), nfiltered=ref["nfiltered"]))


def contract_case(name, seed, alpha, beta, eps):
    # R(mu, lam, P) = sum_{nu, Q} T1(Q, mu, nu) T2(nu, P, Q, lam): two index pairs, the
    # first tensor read through a permuted view, the result stored in a permuted order
    rng = np.random.default_rng(seed)
    nq, nmu, nnu, nP, nlam = 3, 3, 2, 2, 3
    sq, smu, snu, sP, slam = (rng.choice(SIZES, n).astype(np.int32)
                              for n in (nq, nmu, nnu, nP, nlam))
    T1 = int_tensor(rng, [sq, smu, snu], 0.6)
    T2 = int_tensor(rng, [snu, sP, sq, slam], 0.5)
    c1, c2, f1, f2, ro = [2, 0], [0, 2], [1], [1, 3], [0, 2, 1]
    Rin = int_tensor(rng, [smu, slam, sP], 0.3)
    ref = oracle.contract(T(T1), T(T2), c1, c2, f1, f2, ro, T(Rin), alpha, beta, eps)
    return dict(
        name=name,
        cites="Sec. 4 (tensor contraction recast as a block-sparse matrix product)",
        op="contract", c1=c1, c2=c2, f1=f1, f2=f2, result_order=ro,
        alpha=alpha, beta=beta, eps=eps, T1=T1, T2=T2, R_in=Rin,
        expected=dict(index=_ints(ref["index"]), offsets=_ints(ref["offsets"]),
                      data=_ints(ref["data"]), npairs=ref["npairs"],
                      nfiltered=ref["nfiltered"]))


CASES = {
    "multiply_int_filter.json": lambda: multiply_case(
        "mixed 1/2/3/5 blocks, C_in, alpha 2, beta -1, filter eps 6.5", 7, 6, 5, 4,
        "N", "N", 2.0, -1.0, 6.5, 0.3),
    "multiply_int_trans.json": lambda: multiply_case(
        "C = A^T B, tall inner dimension, no filter", 8, 3, 12, 3, "T", "N", 1.0, 0.0, 0.0, 0.0),
    "contract_int_rank4.json": lambda: contract_case(
        "rank-3 x rank-4 over two index pairs, permuted result, R_in, eps 150.5", 9, 1.0, 3.0, 150.5),
}


def main():
    for fname, make in CASES.items():
        case = make()
        with open(os.path.join(HERE, fname), "w") as f:
            json.dump(case, f, separators=(",", ":"))
            f.write("\n")
        e = case["expected"]
        print(fname, len(e["data"]), "values", e.get("nfiltered"), "filtered")


if __name__ == "__main__":
    main()
