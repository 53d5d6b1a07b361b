"""The K-split product's host side (paper Sec. 3.1) on the CPU: K ranges, the cut of a
matrix to a K range, the exchange layout (union pattern, owners, runs, receive tables)
and, with two gloo processes, the pattern gather and the all-to-all.  The partial
products come from the CPU oracle; the owners' fixed-order sums are done here in numpy
from the layout's tables, so what is checked is that the layout sends every element of
every partial product to the right place: the assembled C equals the undivided product
(pattern bit-exact, values within rounding)."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1910_13555_gb300 import ksplit
from paper_1910_13555_gb300.workloads import BSMatrix, tall_skinny

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _small(seed=5, eps=0.0):
    return tall_skinny(seed=seed, nk=600, nmn=30, window=8, p=0.4, kmin=3, kmax=9, eps=eps)


def _cut(M, trans, side, lo, hi):
    r, c, d = ksplit.select_k_range(M.row_sizes, M.col_sizes, M.rows, M.cols, M.data, trans,
                                    side, lo, hi)
    return BSMatrix(M.row_sizes, M.col_sizes, r, c, d)


def _ranges(p, P):
    A, B = p.A, p.B
    ka = ksplit.k_index(A.rows, A.cols, p.transa, "A")
    kb = ksplit.k_index(B.rows, B.cols, p.transb, "B")
    ea = A.row_sizes[A.rows].astype(np.int64) * A.col_sizes[A.cols]
    eb = B.row_sizes[B.rows].astype(np.int64) * B.col_sizes[B.cols]
    ks = A.row_sizes if p.transa == "T" else A.col_sizes
    return ksplit.k_ranges(ka, ea, kb, eb, ks, P)


def _partials(p, P, with_cin=False, alpha=1.0, beta=0.0):
    r = _ranges(p, P)
    parts = []
    for i in range(P):
        Ai = _cut(p.A, p.transa, "A", r[i], r[i + 1])
        Bi = _cut(p.B, p.transb, "B", r[i], r[i + 1])
        Ci = p.C_in if (with_cin and i == 0) else None
        parts.append(oracle.multiply(Ai, Bi, Ci, alpha, beta if i == 0 else 0.0, p.eps,
                                     p.transa, p.transb))
    return r, parts


def _c_sizes(p):
    rs = p.A.col_sizes if p.transa == "T" else p.A.row_sizes
    cs = p.B.row_sizes if p.transb == "T" else p.B.col_sizes
    return rs, cs


def _owner_sum(layout, q, recv):
    """The owner's fixed-order sum, written out from the layout's definition."""
    rows, cols, offs = layout.owned(q)
    out = np.zeros(int(offs[-1]))
    tab = layout.src_off[q]
    for u in range(len(rows)):
        n = int(offs[u + 1] - offs[u])
        acc = None
        for i in range(tab.shape[0]):
            o = int(tab[i, u])
            if o < 0:
                continue
            v = recv[o:o + n]
            acc = v.copy() if acc is None else acc + v
        if acc is not None:
            out[offs[u]:offs[u] + n] = acc
    return out


def _simulate(layout, parts):
    """Each owner's receive buffer: the runs of every partial product, process 0 first."""
    P = len(parts)
    bufs = []
    for q in range(P):
        chunks = []
        for i in range(P):
            start = int(layout.send[i, :q].sum())
            chunks.append(parts[i]["data"][start:start + int(layout.send[i, q])])
        bufs.append(np.concatenate(chunks) if chunks else np.zeros(0))
    return bufs


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_k_ranges_cover_and_balance():
    p = _small()
    for P in (1, 2, 3, 7):
        r = _ranges(p, P)
        K = len(p.A.row_sizes)
        assert r[0] == 0 and r[-1] == K and (np.diff(r) >= 0).all() and len(r) == P + 1
    # uniform work: equal ranges
    r = ksplit.k_ranges(np.arange(100), np.ones(100), np.arange(100), np.ones(100),
                        np.ones(100), 4)
    assert list(r) == [0, 25, 50, 75, 100]


def test_select_k_range_partitions_the_blocks():
    p = _small()
    r = _ranges(p, 3)
    got = [_cut(p.A, "T", "A", r[i], r[i + 1]) for i in range(3)]
    assert sum(len(g.rows) for g in got) == len(p.A.rows)
    assert np.array_equal(np.concatenate([g.data for g in got]), p.A.data)  # row ranges
    for i, g in enumerate(got):
        assert ((g.rows >= r[i]) & (g.rows < r[i + 1])).all()
    # K along block columns (op = N): blocks keep CSR order, data follows its blocks
    Bt = _cut(p.A, "N", "A", 3, 11)
    assert ((Bt.cols >= 3) & (Bt.cols < 11)).all()
    lens = p.A.row_sizes[p.A.rows].astype(np.int64) * p.A.col_sizes[p.A.cols]
    offs = np.concatenate(([0], np.cumsum(lens)))
    keep = np.nonzero((p.A.cols >= 3) & (p.A.cols < 11))[0]
    ref = np.concatenate([p.A.data[offs[b]:offs[b + 1]] for b in keep])
    assert np.array_equal(Bt.data, ref)


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_layout_assembles_the_undivided_product(P):
    p = _small(eps=10.0)
    full = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb)
    r, parts = _partials(p, P)
    # the filter acts on single block products: the split keeps the same products
    assert sum(x["nfiltered"] for x in parts) == full["nfiltered"] > 0
    rs, cs = _c_sizes(p)
    lay = ksplit.exchange_layout([(x["rows"], x["cols"]) for x in parts], rs, cs)
    assert np.array_equal(lay.rows, full["rows"]) and np.array_equal(lay.cols, full["cols"])
    assert np.array_equal(lay.offsets[:-1], full["offsets"])
    assert lay.owner[0] == 0 and lay.owner[-1] == len(lay.rows)
    for i in range(P):
        assert lay.send[i].sum() == len(parts[i]["data"])
    bufs = _simulate(lay, parts)
    got = np.concatenate([_owner_sum(lay, q, bufs[q]) for q in range(P)])
    assert _rel(got, full["data"]) <= 1e-13
    # fixed order: the same as adding the partial products scattered into C, 0 first
    ref = None
    for x in parts:
        dense = np.zeros(int(lay.offsets[-1]))
        hit = np.zeros(int(lay.offsets[-1]), bool)
        ui = np.searchsorted(lay.rows.astype(np.int64) * 10 ** 6 + lay.cols,
                             x["rows"].astype(np.int64) * 10 ** 6 + x["cols"])
        for j, u in enumerate(ui):
            n = int(lay.offsets[u + 1] - lay.offsets[u])
            o = int(x["offsets"][j])
            dense[lay.offsets[u]:lay.offsets[u] + n] = x["data"][o:o + n]
            hit[lay.offsets[u]:lay.offsets[u] + n] = True
        ref = np.where(hit, dense, 0.0) if ref is None else np.where(hit, ref + dense, ref)
    assert np.array_equal(got, ref)


def test_layout_with_cin_on_process_zero():
    rng = np.random.default_rng(9)
    p = _small(seed=6)
    rs, cs = _c_sizes(p)
    full0 = oracle.multiply(p.A, p.B, None, 1.0, 0.0, 0.0, p.transa, p.transb)
    keep = rng.random(len(full0["rows"])) < 0.4
    r_in = full0["rows"][keep]
    c_in = full0["cols"][keep]
    # plus blocks no product reaches
    extra = [(a, b) for a, b in zip(rng.integers(0, len(rs), 15), rng.integers(0, len(cs), 15))]
    pairs = sorted(set(zip(r_in.tolist(), c_in.tolist())) | set(extra))
    r_in = np.array([a for a, _ in pairs], np.int32)
    c_in = np.array([b for _, b in pairs], np.int32)
    d_in = rng.uniform(-1, 1, int((rs[r_in].astype(np.int64) * cs[c_in]).sum()))
    from paper_1910_13555_gb300.workloads import Problem
    q = Problem(p.A, p.B, BSMatrix(rs, cs, r_in, c_in, d_in), 0.5, -2.0, 0.0, "T", "N")
    full = oracle.multiply(q.A, q.B, q.C_in, q.alpha, q.beta, 0.0, "T", "N")
    _, parts = _partials(q, 3, with_cin=True, alpha=q.alpha, beta=q.beta)
    lay = ksplit.exchange_layout([(x["rows"], x["cols"]) for x in parts], rs, cs)
    assert np.array_equal(lay.rows, full["rows"]) and np.array_equal(lay.cols, full["cols"])
    bufs = _simulate(lay, parts)
    got = np.concatenate([_owner_sum(lay, k, bufs[k]) for k in range(3)])
    assert _rel(got, full["data"]) <= 1e-13


def test_layout_rejects_unsorted_pattern_and_handles_empty_parts():
    with pytest.raises(ValueError):
        ksplit.exchange_layout([(np.array([1, 0]), np.array([0, 0]))], np.ones(3, np.int32),
                               np.ones(3, np.int32))
    e = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    lay = ksplit.exchange_layout([e, (np.array([0, 2], np.int32), np.array([1, 0], np.int32)), e],
                                 np.array([2, 3, 4], np.int32), np.array([5, 6], np.int32))
    assert lay.send.sum() == 2 * 6 + 4 * 5
    assert list(lay.offsets) == [0, 12, 32]
    assert (lay.send[0] == 0).all() and (lay.send[2] == 0).all()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np, torch, torch.distributed as dist
import test_ksplit as T
from paper_1910_13555_gb300 import ksplit
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
p = T._small(eps=10.0)
r, parts = T._partials(p, world)
mine = parts[rank]                      # this process's partial product
rs, cs = T._c_sizes(p)
pats = ksplit.gather_patterns(mine["rows"], mine["cols"])
lay = ksplit.exchange_layout(pats, rs, cs)
recv = ksplit.exchange(torch.as_tensor(mine["data"]), lay).numpy()
out = T._owner_sum(lay, rank, recv)
rows, cols, offs = lay.owned(rank)
np.save(os.environ["OUT"], np.concatenate([[len(rows)], rows, cols, out]))
dist.destroy_process_group()
"""


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_processes_gather_exchange_and_sum(tmp_path, world):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OUT=str(tmp_path / f"r{r}.npy"))
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER.format(root=ROOT)],
                                      env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    for pr in procs:
        _, err = pr.communicate(timeout=180)
        assert pr.returncode == 0, err
    p = _small(eps=10.0)
    full = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb)
    rows, cols, data = [], [], []
    for r in range(world):
        a = np.load(tmp_path / f"r{r}.npy")
        n = int(a[0])
        rows.append(a[1:1 + n])
        cols.append(a[1 + n:1 + 2 * n])
        data.append(a[1 + 2 * n:])
    assert np.array_equal(np.concatenate(rows), full["rows"])
    assert np.array_equal(np.concatenate(cols), full["cols"])
    assert _rel(np.concatenate(data), full["data"]) <= 1e-13
    assert all(len(x) > 0 for x in rows)  # every process owns a share


def _rank3_small():
    from paper_1910_13555_gb300.workloads import rank3
    return rank3(nP=120, sP=6, nao=40, window=6, p=0.4)


def test_contraction_split_over_the_auxiliary_index():
    """A rank-3 contraction R(mu, lam) = sum_{P, nu} T(P, mu, nu) U(P, nu, lam) split over
    P among 3 processes (paper Sec. 4's long contracted index): the oracle's partial
    contractions, their folds, the layout and the owners' sums assemble the undivided
    result (index bit-exact, values within rounding); fold and unfold are inverses."""
    w = _rank3_small()
    full = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    nP = len(w.T1.block_sizes[0])
    bounds = [0, nP // 3, 2 * nP // 3, nP]
    parts, pats = [], []
    rsz = ksplit.result_block_sizes(w.T1.block_sizes, w.T2.block_sizes, w.f1, w.f2,
                                    w.result_order)
    from paper_1910_13555_gb300.workloads import BSTensor
    for i in range(3):
        i1, d1 = ksplit.select_tensor_range(w.T1.block_sizes, w.T1.index, w.T1.data,
                                            w.c1[0], bounds[i], bounds[i + 1])
        i2, d2 = ksplit.select_tensor_range(w.T2.block_sizes, w.T2.index, w.T2.data,
                                            w.c2[0], bounds[i], bounds[i + 1])
        r = oracle.contract(BSTensor(w.T1.block_sizes, i1, d1), BSTensor(w.T2.block_sizes, i2, d2),
                            w.c1, w.c2, w.f1, w.f2, w.result_order)
        rows, cols, row_sizes, col_sizes = ksplit.tensor_fold(r["index"], rsz)
        assert np.array_equal(ksplit.tensor_unfold(rows, cols, rsz), r["index"])
        parts.append(r)
        pats.append((rows, cols))
    lay = ksplit.exchange_layout(pats, row_sizes, col_sizes)
    assert np.array_equal(ksplit.tensor_unfold(lay.rows, lay.cols, rsz), full["index"])
    assert np.array_equal(lay.offsets[:-1], full["offsets"])
    bufs = _simulate(lay, parts)
    got = np.concatenate([_owner_sum(lay, q, bufs[q]) for q in range(3)])
    assert _rel(got, full["data"]) <= 1e-13


@pytest.mark.parametrize("rank", [1, 2, 3, 4])
def test_tensor_fold_roundtrip_and_order(rank):
    """tensor_fold: rows in mixed radix over the modes but the last (mode 0 slowest), so
    lexicographic tuple order is CSR order; row sizes are the products of the modes'
    sizes; tensor_unfold inverts it."""
    rng = np.random.default_rng(rank)
    sizes = [rng.integers(1, 6, rng.integers(2, 6)) for _ in range(rank)]
    grid = np.stack(np.meshgrid(*[np.arange(len(s)) for s in sizes], indexing="ij"), -1)
    idx = grid.reshape(-1, rank)[rng.random(int(np.prod([len(s) for s in sizes]))) < 0.5]
    rows, cols, row_sizes, col_sizes = ksplit.tensor_fold(idx, sizes)
    assert np.array_equal(ksplit.tensor_unfold(rows, cols, sizes), idx)
    key = rows.astype(np.int64) * len(col_sizes) + cols
    assert (np.diff(key) > 0).all()  # lexicographic tuples -> increasing (row, col)
    lens = np.ones(len(idx), np.int64)
    for d, s in enumerate(sizes):
        lens *= s[idx[:, d]]
    assert np.array_equal(row_sizes[rows] * col_sizes[cols], lens)


def test_result_block_sizes_follow_result_order():
    s1 = [np.array([1, 2]), np.array([3]), np.array([4, 5, 6])]
    s2 = [np.array([7]), np.array([8, 9])]
    out = ksplit.result_block_sizes(s1, s2, f1=[1, 2], f2=[1], result_order=[2, 0, 1])
    assert [list(x) for x in out] == [[8, 9], [3], [4, 5, 6]]
