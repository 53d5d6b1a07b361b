"""Seeded synthetic inputs shaped like the paper's workloads (input generation only).

This module holds no arithmetic of the method: it draws block sizes, block patterns
and element values with ``numpy.random.default_rng(seed)`` and packs them in the
canonical layout (blocks in (row, col) order -- lexicographic tuple order for
tensors -- each block row-major).  Both the CUDA library's tests/benchmarks and the
CPU oracle's tests take their inputs from here; neither side's code lives here.

Shapes follow the paper: chemically sized blocks from an atom-centred basis
(Sec. 1: blocked sparsity with chemically motivated block sizes), occupancies between
0.01 % and 10 % (Sec. 1 and its related-work paragraph), tall-and-skinny products
with K >> M, N (Sec. 3, Sec. 4: a rank-3 tensor folds two modes into one matrix
dimension).  The five named workloads are:

  plain        40x40 blocks of size 5, Bernoulli(0.10) patterns, U[-1,1], eps = 0
  banded       4000x4000 blocks, sizes {5:.4, 13:.4, 23:.2}, banded ~1 % occupancy
               (kept w.p. c*exp(-|i-j|/200), c = 0.01/mean), entries
               N(0,1)*exp(-|i-j|/50), eps = 1e-8
  tall_skinny  A, B 100000x400 blocks, row sizes U{20..50}, column sizes {5,13};
               windowed locality giving 0.5 % occupancy and a ~28 % dense C = A^T B
  batched      64 square problems, n = floor(exp U[ln 200, ln 3000]) blocks, occupancy
               exp U[ln 1e-3, ln 1e-1], sizes {5,13,23}, U[-1,1] x 10^-U[0,8] per block,
               eps = 1e-10; problem p draws from default_rng((seed, p))
  rank3        T(P,mu,nu), U(P,nu,lam), P: 2000 blocks of 30, mu/nu/lam: 1000 blocks of
               {5,13}; windowed 0.01 % occupancy (~2e5 blocks per tensor)

Every generator takes scale arguments so that the tests can draw the same recipe at
sizes the CPU oracle finishes in seconds.

The eps guard: with a filter eps > 0 the generators rescale (by 1.01, up to 8 times)
every A block whose norm product with some B partner lies within 1e-6 relative of eps,
so no filter decision depends on how a norm is rounded.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SIZES_5_13_23 = (np.array([5, 13, 23], np.int32), np.array([0.4, 0.4, 0.2]))


@dataclass
class BSMatrix:
    """Block-sparse matrix in canonical CSR block order."""
    row_sizes: np.ndarray   # int32 [nbr]
    col_sizes: np.ndarray   # int32 [nbc]
    rows: np.ndarray        # int32 [nblocks], ascending (row, col)
    cols: np.ndarray        # int32 [nblocks]
    data: np.ndarray        # float64, blocks packed in order, each row-major

    @property
    def nblocks(self) -> int:
        return len(self.rows)

    @property
    def block_lens(self) -> np.ndarray:
        return (self.row_sizes[self.rows].astype(np.int64) *
                self.col_sizes[self.cols].astype(np.int64))

    @property
    def offsets(self) -> np.ndarray:
        lens = self.block_lens
        off = np.zeros(len(lens), np.int64)
        if len(lens) > 1:
            np.cumsum(lens[:-1], out=off[1:])
        return off


@dataclass
class BSTensor:
    """Block-sparse tensor: per-mode block sizes, tuples in lexicographic order."""
    block_sizes: list       # list of int32 arrays, one per mode
    index: np.ndarray       # int32 [nblocks, rank], lexicographic
    data: np.ndarray        # float64, blocks packed in order, each row-major

    @property
    def rank(self) -> int:
        return len(self.block_sizes)

    @property
    def nblocks(self) -> int:
        return self.index.shape[0]

    @property
    def block_lens(self) -> np.ndarray:
        lens = np.ones(self.nblocks, np.int64)
        for d, s in enumerate(self.block_sizes):
            lens *= np.asarray(s, np.int64)[self.index[:, d]]
        return lens

    @property
    def offsets(self) -> np.ndarray:
        lens = self.block_lens
        off = np.zeros(len(lens), np.int64)
        if len(lens) > 1:
            np.cumsum(lens[:-1], out=off[1:])
        return off


@dataclass
class Problem:
    """A multiply C = alpha*op(A)*op(B) + beta*C_in with its filter."""
    A: BSMatrix
    B: BSMatrix
    C_in: BSMatrix | None = None
    alpha: float = 1.0
    beta: float = 0.0
    eps: float = 0.0
    transa: str = "N"
    transb: str = "N"
    name: str = ""
    meta: dict = field(default_factory=dict)


@dataclass
class Contraction:
    T1: BSTensor
    T2: BSTensor
    c1: list
    c2: list
    f1: list
    f2: list
    result_order: list | None = None
    R_in: BSTensor | None = None
    alpha: float = 1.0
    beta: float = 0.0
    eps: float = 0.0
    name: str = ""
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------------
# primitives


def draw_sizes(rng, n, choices=SIZES_5_13_23):
    vals, probs = choices
    return rng.choice(vals, size=n, p=probs).astype(np.int32)


def _sorted_pattern(rows, cols):
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    order = np.lexsort((cols, rows))
    return rows[order].astype(np.int32), cols[order].astype(np.int32)


def make_matrix(rng, row_sizes, col_sizes, rows, cols, dist="uniform", scale=None):
    """Pack a matrix with the given pattern; values U[-1,1] or N(0,1), times an
    optional per-block scale (array over blocks)."""
    rows, cols = _sorted_pattern(rows, cols)
    row_sizes = np.asarray(row_sizes, np.int32)
    col_sizes = np.asarray(col_sizes, np.int32)
    lens = row_sizes[rows].astype(np.int64) * col_sizes[cols].astype(np.int64)
    n = int(lens.sum())
    if dist == "uniform":
        data = rng.uniform(-1.0, 1.0, n)
    elif dist == "normal":
        data = rng.standard_normal(n)
    else:
        raise ValueError(dist)
    m = BSMatrix(row_sizes, col_sizes, rows, cols, data)
    if scale is not None:
        s = scale(rows, cols) if callable(scale) else np.asarray(scale)
        m.data *= np.repeat(np.asarray(s, np.float64), lens)
    return m


def bernoulli_pattern(rng, nbr, nbc, occ):
    """iid Bernoulli(occ) block pattern, drawn row-chunked to bound memory."""
    rows, cols = [], []
    chunk = max(1, (1 << 24) // max(nbc, 1))
    for r0 in range(0, nbr, chunk):
        r1 = min(nbr, r0 + chunk)
        keep = rng.random((r1 - r0, nbc)) < occ
        r, c = np.nonzero(keep)
        rows.append(r + r0)
        cols.append(c)
    if not rows:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.concatenate(rows).astype(np.int32), np.concatenate(cols).astype(np.int32)


def _np_block_norms(m: BSMatrix) -> np.ndarray:
    lens = m.block_lens
    if len(lens) == 0:
        return np.zeros(0)
    sq = np.add.reduceat(m.data * m.data, m.offsets) if m.data.size else np.zeros(len(lens))
    return np.sqrt(sq)


def eps_guard(A: BSMatrix, B: BSMatrix, eps: float, transa="N", transb="N", rel=1e-6,
              tries=8):
    """Rescale A blocks (x1.01) until no candidate product norm is within rel*eps of eps."""
    if eps <= 0.0:
        return 0
    # inner index of each stored block of op(A) and op(B)
    ka = A.rows if transa in "Tt" else A.cols
    kb = B.cols if transb in "Tt" else B.rows
    nk = len(A.row_sizes) if transa in "Tt" else len(A.col_sizes)
    ob = np.argsort(kb, kind="stable")
    ptr = np.zeros(nk + 1, np.int64)
    np.add.at(ptr, np.asarray(kb, np.int64) + 1, 1)
    ptr = np.cumsum(ptr)
    cnt = ptr[ka + 1] - ptr[ka]
    a_rep = np.repeat(np.arange(A.nblocks), cnt)
    starts = np.repeat(ptr[ka], cnt)
    within = np.arange(len(a_rep)) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    b_idx = ob[starts + within]
    lens = A.block_lens
    offs = A.offsets
    rescaled = 0
    for _ in range(tries):
        na = _np_block_norms(A)
        nb = _np_block_norms(B)
        pn = na[a_rep] * nb[b_idx]
        bad = np.unique(a_rep[np.abs(pn - eps) <= rel * eps])
        if len(bad) == 0:
            return rescaled
        for b in bad:
            A.data[offs[b]:offs[b] + lens[b]] *= 1.01
        rescaled += len(bad)
    raise RuntimeError("eps guard did not converge")


# ----------------------------------------------------------------------------------
# the five workloads


def plain(seed=1001, nb=40, size=5, occ=0.10) -> Problem:
    """Uniform-size block-sparse C = A*B, Bernoulli pattern, eps = 0, beta = 0."""
    rng = np.random.default_rng(seed)
    sz = np.full(nb, size, np.int32)
    ra, ca = bernoulli_pattern(rng, nb, nb, occ)
    A = make_matrix(rng, sz, sz, ra, ca)
    rb, cb = bernoulli_pattern(rng, nb, nb, occ)
    B = make_matrix(rng, sz, sz, rb, cb)
    return Problem(A, B, None, 1.0, 0.0, 0.0, name=f"plain nb={nb} size={size} occ={occ}")


def banded_pattern(rng, nb, occ=0.01, decay=200.0):
    """Keep (i, j) with probability c*exp(-|i-j|/decay), c chosen for mean occ."""
    d = np.arange(nb)
    mean = np.mean(np.exp(-np.abs(d[:, None] - d[None, :]) / decay)) if nb <= 4096 else None
    if mean is None:
        s = 0.0
        for i in range(0, nb, 512):
            s += np.exp(-np.abs(d[i:i + 512, None] - d[None, :]) / decay).sum()
        mean = s / (nb * nb)
    c = min(1.0, occ / mean)
    rows, cols = [], []
    chunk = max(1, (1 << 23) // max(nb, 1))
    for r0 in range(0, nb, chunk):
        r1 = min(nb, r0 + chunk)
        p = c * np.exp(-np.abs(d[r0:r1, None] - d[None, :]) / decay)
        r, cc = np.nonzero(rng.random((r1 - r0, nb)) < p)
        rows.append(r + r0)
        cols.append(cc)
    return np.concatenate(rows).astype(np.int32), np.concatenate(cols).astype(np.int32), c


def banded(seed=1002, nb=4000, occ=0.01, decay=200.0, value_decay=50.0, eps=1e-8,
           sizes=SIZES_5_13_23, block_mkn=None) -> Problem:
    """Banded block-sparse product with mixed 5/13/23 blocks and a norm filter.
    block_mkn = (m, k, n) gives every block row of A the size m, every inner block k and
    every block column of B the size n instead (a single (m, n, k) stack)."""
    rng = np.random.default_rng(seed)
    sz = draw_sizes(rng, nb, sizes)
    if block_mkn is None:
        sm = sk = sn = sz
    else:
        sm, sk, sn = (np.full(nb, v, np.int32) for v in block_mkn)

    def vscale(r, c):
        return np.exp(-np.abs(r.astype(np.float64) - c) / value_decay)

    ra, ca, c = banded_pattern(rng, nb, occ, decay)
    A = make_matrix(rng, sm, sk, ra, ca, dist="normal", scale=vscale)
    rb, cb, _ = banded_pattern(rng, nb, occ, decay)
    B = make_matrix(rng, sk, sn, rb, cb, dist="normal", scale=vscale)
    n = eps_guard(A, B, eps)
    return Problem(A, B, None, 1.0, 0.0, eps, name=f"banded nb={nb}",
                   meta=dict(keep_scale=c, guard_rescaled=n))


def tall_skinny(seed=1003, nk=100000, nmn=400, window=60, p=1.0 / 30, kmin=20, kmax=50,
                eps=0.0) -> Problem:
    """C(mu,nu) = sum_{P lam} A(P lam, mu) B(P lam, nu): C = A^T B with K >> M, N.

    Row block r (a (P, lam) pair) has a centre c_r ~ U[0, nmn); columns in the circular
    window [c_r, c_r + window) are kept with probability p, the same centre for A and B.
    """
    rng = np.random.default_rng(seed)
    ksz = rng.integers(kmin, kmax + 1, nk).astype(np.int32)
    msz = rng.choice(np.array([5, 13], np.int32), nmn).astype(np.int32)
    centre = rng.integers(0, nmn, nk)

    def pattern():
        keep = rng.random((nk, window)) < p
        r, w = np.nonzero(keep)
        return r.astype(np.int32), ((centre[r] + w) % nmn).astype(np.int32)

    ra, ca = pattern()
    A = make_matrix(rng, ksz, msz, ra, ca)
    rb, cb = pattern()
    B = make_matrix(rng, ksz, msz, rb, cb)
    eps_guard(A, B, eps, transa="T")
    return Problem(A, B, None, 1.0, 0.0, eps, transa="T", name=f"tall_skinny nk={nk} nmn={nmn}")


def rect_case2(seed=1006, nm=20000, nk=400, window=60, p=1.0 / 30, bwin=20, bp=0.5, kmin=20,
               kmax=50, eps=0.0) -> Problem:
    """C(P lam, nu) = sum_mu A(P lam, mu) B(mu, nu): the rectangular case S_B << S_A, S_C
    (a small B between a tall A and a tall C).

    A: nm x nk blocks, row blocks of U{kmin..kmax}, columns {5, 13}; row block r keeps the
    columns of the circular window [c_r, c_r + window) w.p. p (c_r ~ U[0, nk)).
    B: nk x nk blocks {5, 13}; (mu, nu) kept w.p. bp when (nu - mu) mod nk < bwin."""
    rng = np.random.default_rng(seed)
    msz = rng.integers(kmin, kmax + 1, nm).astype(np.int32)
    ksz = rng.choice(np.array([5, 13], np.int32), nk).astype(np.int32)
    centre = rng.integers(0, nk, nm)
    keep = rng.random((nm, window)) < p
    r, w = np.nonzero(keep)
    A = make_matrix(rng, msz, ksz, r, (centre[r] + w) % nk)
    keep_b = rng.random((nk, bwin)) < bp
    mu, d = np.nonzero(keep_b)
    B = make_matrix(rng, ksz, ksz, mu, (mu + d) % nk)
    eps_guard(A, B, eps)
    return Problem(A, B, None, 1.0, 0.0, eps, name=f"rect_case2 nm={nm} nk={nk}")


def batched(seed=1004, nprob=64, nmin=200, nmax=3000, occ_min=1e-3, occ_max=1e-1,
            eps=1e-10, sizes=SIZES_5_13_23):
    """Independent square problems of log-uniform size and occupancy."""
    probs = []
    for p in range(nprob):
        rng = np.random.default_rng((seed, p))
        n = int(np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        occ = float(np.exp(rng.uniform(np.log(occ_min), np.log(occ_max))))
        sz = draw_sizes(rng, n, sizes)

        def bscale(r, c, rng=rng):
            return 10.0 ** (-rng.uniform(0.0, 8.0, len(r)))

        ra, ca = bernoulli_pattern(rng, n, n, occ)
        A = make_matrix(rng, sz, sz, ra, ca, scale=bscale)
        rb, cb = bernoulli_pattern(rng, n, n, occ)
        B = make_matrix(rng, sz, sz, rb, cb, scale=bscale)
        eps_guard(A, B, eps)
        probs.append(Problem(A, B, None, 1.0, 0.0, eps, name=f"batched[{p}] n={n} occ={occ:.2e}",
                             meta=dict(n=n, occ=occ)))
    return probs


def _tensor(rng, block_sizes, index, dist="uniform"):
    index = np.asarray(index, np.int32)
    order = np.lexsort(tuple(index[:, d] for d in range(index.shape[1] - 1, -1, -1)))
    index = np.ascontiguousarray(index[order])
    lens = np.ones(len(index), np.int64)
    for d, s in enumerate(block_sizes):
        lens *= np.asarray(s, np.int64)[index[:, d]]
    n = int(lens.sum())
    data = rng.uniform(-1.0, 1.0, n) if dist == "uniform" else rng.standard_normal(n)
    return BSTensor([np.asarray(s, np.int32) for s in block_sizes], index, data)


def rank3(seed=1005, nP=2000, sP=30, nao=1000, window=20, p=0.25, eps=0.0) -> Contraction:
    """R(mu,lam) = sum_{P,nu} T(P,mu,nu) U(P,nu,lam) with windowed locality.

    Each P has a centre c_P; T(P,mu,nu) is kept w.p. p when mu and nu both lie in the
    circular window [c_P, c_P + window) of AO blocks, and likewise U(P,nu,lam)."""
    rng = np.random.default_rng(seed)
    psz = np.full(nP, sP, np.int32)
    aosz = rng.choice(np.array([5, 13], np.int32), nao).astype(np.int32)
    centre = rng.integers(0, nao, nP)

    def pattern():
        keep = rng.random((nP, window, window)) < p
        P, a, b = np.nonzero(keep)
        return np.stack([P, (centre[P] + a) % nao, (centre[P] + b) % nao], 1)

    T = _tensor(rng, [psz, aosz, aosz], pattern())
    U = _tensor(rng, [psz, aosz, aosz], pattern())
    return Contraction(T, U, c1=[0, 2], c2=[0, 1], f1=[1], f2=[2], result_order=None,
                       eps=eps, name=f"rank3 nP={nP} nao={nao}")


def rank4(seed=1007, nP=400, sP=30, nao=400, window=8, p4=0.04, p3=0.25, eps=0.0) -> Contraction:
    """R(mu, sig, lam) = sum_{P, nu} V(P, mu, nu, lam) U(P, nu, sig): a rank-4 tensor
    contracted with a rank-3 one over two index pairs, the free modes of V not adjacent
    (its matrix view needs a permuted copy) and the result modes reordered.

    Each P has a centre c_P; V(P, mu, nu, lam) is kept w.p. p4 when mu, nu, lam all lie
    in the circular window [c_P, c_P + window) of AO blocks, U(P, nu, sig) w.p. p3."""
    rng = np.random.default_rng(seed)
    psz = np.full(nP, sP, np.int32)
    aosz = rng.choice(np.array([5, 13], np.int32), nao).astype(np.int32)
    centre = rng.integers(0, nao, nP)
    keep = rng.random((nP, window, window, window)) < p4
    P, a, b, c = np.nonzero(keep)
    V = _tensor(rng, [psz, aosz, aosz, aosz],
                np.stack([P, (centre[P] + a) % nao, (centre[P] + b) % nao, (centre[P] + c) % nao], 1))
    keep = rng.random((nP, window, window)) < p3
    P, a, b = np.nonzero(keep)
    U = _tensor(rng, [psz, aosz, aosz], np.stack([P, (centre[P] + a) % nao, (centre[P] + b) % nao], 1))
    return Contraction(V, U, c1=[0, 2], c2=[0, 1], f1=[1, 3], f2=[2], result_order=[0, 2, 1],
                       eps=eps, name=f"rank4 nP={nP} nao={nao}")


def sign_matrix(seed=1008, nb=2000, width=6, p=0.5, coupling=0.1, gap=0.3,
                sizes=SIZES_5_13_23) -> BSMatrix:
    """A symmetric block-sparse matrix for the matrix-sign iteration (paper Sec. 2, the
    linear-scaling DFT use of chained filtered multiplies), scaled so that its spectrum
    lies in [-1, 1] away from 0.

    Diagonal blocks Q diag(+-U[gap, 1]) Q^T (Q random orthogonal); off-diagonal blocks
    (i, j), 0 < j - i <= width, kept w.p. p with N(0,1) entries times coupling/sqrt(n_i n_j),
    mirrored to (j, i) transposed; the whole matrix divided by its largest absolute row
    sum (a bound on the spectral radius)."""
    rng = np.random.default_rng(seed)
    sz = draw_sizes(rng, nb, sizes)
    rows, cols, blocks = [], [], {}
    for i in range(nb):
        n = int(sz[i])
        q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = rng.uniform(gap, 1.0, n) * rng.choice([-1.0, 1.0], n)
        blocks[(i, i)] = (q * lam) @ q.T
        for j in range(i + 1, min(nb, i + width + 1)):
            if rng.random() < p:
                m = int(sz[j])
                b = rng.standard_normal((n, m)) * coupling / np.sqrt(n * m)
                blocks[(i, j)] = b
                blocks[(j, i)] = b.T.copy()
    keys = sorted(blocks)
    rows = np.array([k[0] for k in keys], np.int32)
    cols = np.array([k[1] for k in keys], np.int32)
    rowsum = np.zeros(int(sz.sum()))
    starts = np.concatenate([[0], np.cumsum(sz)])
    for (i, j) in keys:
        rowsum[starts[i]:starts[i + 1]] += np.abs(blocks[(i, j)]).sum(1)
    scale = 1.0 / rowsum.max()
    data = np.concatenate([blocks[k].ravel() * scale for k in keys])
    return BSMatrix(sz, sz, rows, cols, data)


def random_tensor(rng, nblk, sizes, occ, dist="uniform"):
    """iid Bernoulli(occ) tensor with per-mode block sizes (small test tensors)."""
    rank = len(nblk)
    grids = np.stack(np.meshgrid(*[np.arange(n) for n in nblk], indexing="ij"), -1)
    tuples = grids.reshape(-1, rank)
    keep = rng.random(len(tuples)) < occ
    bs = [np.asarray(sizes[d], np.int32) for d in range(rank)]
    return _tensor(rng, bs, tuples[keep], dist)
