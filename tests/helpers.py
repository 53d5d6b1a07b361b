"""Test-side helpers: densify block-sparse inputs and brute-force references.

These are independent restatements used to pin the oracle (dense numpy products,
np.einsum, explicit Python loops); they share no code with the oracle or the library.
"""
from __future__ import annotations

import numpy as np

from paper_1910_13555_gb300.workloads import BSMatrix, BSTensor


def starts(sizes):
    s = np.zeros(len(sizes) + 1, np.int64)
    np.cumsum(np.asarray(sizes, np.int64), out=s[1:])
    return s


def densify(m: BSMatrix) -> np.ndarray:
    rs, cs = starts(m.row_sizes), starts(m.col_sizes)
    D = np.zeros((rs[-1], cs[-1]))
    off = 0
    for b in range(m.nblocks):
        i, j = m.rows[b], m.cols[b]
        r, c = m.row_sizes[i], m.col_sizes[j]
        D[rs[i]:rs[i] + r, cs[j]:cs[j] + c] = m.data[off:off + r * c].reshape(r, c)
        off += r * c
    return D


def pattern_dense(nbr, nbc, rows, cols):
    P = np.zeros((nbr, nbc), bool)
    P[np.asarray(rows), np.asarray(cols)] = True
    return P


def block_of(m: BSMatrix, b: int) -> np.ndarray:
    off = m.offsets[b]
    r, c = m.row_sizes[m.rows[b]], m.col_sizes[m.cols[b]]
    return m.data[off:off + r * c].reshape(r, c)


def transpose_matrix(m: BSMatrix) -> BSMatrix:
    """Stored transpose: block (i,j) -> (j,i) with transposed data, re-packed."""
    order = np.lexsort((m.rows, m.cols))
    data = np.concatenate([block_of(m, b).T.ravel() for b in order]) if len(order) else np.zeros(0)
    return BSMatrix(m.col_sizes.copy(), m.row_sizes.copy(), m.cols[order].copy(),
                    m.rows[order].copy(), data)


def from_result(res, row_sizes, col_sizes) -> BSMatrix:
    return BSMatrix(np.asarray(row_sizes, np.int32), np.asarray(col_sizes, np.int32),
                    res["rows"], res["cols"], res["data"])


def random_matrix(rng, row_sizes, col_sizes, occ, dist="uniform"):
    row_sizes = np.asarray(row_sizes, np.int32)
    col_sizes = np.asarray(col_sizes, np.int32)
    keep = rng.random((len(row_sizes), len(col_sizes))) < occ
    r, c = np.nonzero(keep)
    lens = row_sizes[r].astype(np.int64) * col_sizes[c]
    n = int(lens.sum())
    data = rng.uniform(-1, 1, n) if dist == "uniform" else rng.standard_normal(n)
    return BSMatrix(row_sizes, col_sizes, r.astype(np.int32), c.astype(np.int32), data)


def brute_multiply(A, B, C_in, alpha, beta, eps, transa="N", transb="N"):
    """Block-by-block triple loop in Python with numpy per-block norms and products.

    Returns (dict (i,j) -> dense block, set of kept (i,j,k), filtered count)."""
    Ab = {}
    for b in range(A.nblocks):
        x = block_of(A, b)
        i, k = (A.rows[b], A.cols[b]) if transa == "N" else (A.cols[b], A.rows[b])
        Ab[(int(i), int(k))] = x if transa == "N" else x.T
    Bb = {}
    for b in range(B.nblocks):
        x = block_of(B, b)
        k, j = (B.rows[b], B.cols[b]) if transb == "N" else (B.cols[b], B.rows[b])
        Bb[(int(k), int(j))] = x if transb == "N" else x.T
    out = {}
    kept = set()
    nfilt = 0
    for (i, k), a in Ab.items():
        for (k2, j), b in Bb.items():
            if k2 != k:
                continue
            if np.linalg.norm(a) * np.linalg.norm(b) >= eps:
                kept.add((i, j, k))
                out[(i, j)] = out.get((i, j), 0.0) + a @ b
            else:
                nfilt += 1
    res = {}
    for key, v in out.items():
        res[key] = alpha * v
    if C_in is not None:
        for b in range(C_in.nblocks):
            key = (int(C_in.rows[b]), int(C_in.cols[b]))
            cb = block_of(C_in, b)
            base = res.get(key, np.zeros_like(cb))
            res[key] = base + (beta * cb if beta != 0.0 else 0.0)
    return res, kept, nfilt


def tensor_dense(t: BSTensor) -> np.ndarray:
    st = [starts(s) for s in t.block_sizes]
    D = np.zeros(tuple(int(s[-1]) for s in st))
    offs = t.offsets
    lens = t.block_lens
    for b in range(t.nblocks):
        tup = t.index[b]
        shape = tuple(int(t.block_sizes[d][tup[d]]) for d in range(t.rank))
        sl = tuple(slice(st[d][tup[d]], st[d][tup[d]] + shape[d]) for d in range(t.rank))
        D[sl] = t.data[offs[b]:offs[b] + lens[b]].reshape(shape)
    return D


def tensor_from_result(res, block_sizes) -> BSTensor:
    return BSTensor([np.asarray(s, np.int32) for s in block_sizes], res["index"], res["data"])


def tensor_block_mask(t: BSTensor) -> np.ndarray:
    st = [starts(s) for s in t.block_sizes]
    M = np.zeros(tuple(int(s[-1]) for s in st), bool)
    for b in range(t.nblocks):
        tup = t.index[b]
        sl = tuple(slice(st[d][tup[d]], st[d][tup[d] + 1]) for d in range(t.rank))
        M[sl] = True
    return M


def einsum_spec(r1, r2, c1, c2, f1, f2, result_order):
    letters = "abcdefghijklmnop"
    s1 = [None] * r1
    s2 = [None] * r2
    nxt = 0
    for a, b in zip(c1, c2):
        s1[a] = s2[b] = letters[nxt]
        nxt += 1
    free = []
    for a in f1:
        s1[a] = letters[nxt]
        free.append(letters[nxt])
        nxt += 1
    for b in f2:
        s2[b] = letters[nxt]
        free.append(letters[nxt])
        nxt += 1
    ro = result_order if result_order is not None else list(range(len(free)))
    out = "".join(free[r] for r in ro)
    return f"{''.join(s1)},{''.join(s2)}->{out}"
