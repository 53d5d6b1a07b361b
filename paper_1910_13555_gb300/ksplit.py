"""K-split product over several processes, one GPU each (paper Sec. 3.1).

When C is much smaller than A and B (a tall-skinny C = A^T B with K >> M, N), the inner
block dimension K is divided among the P processes of a group: process i holds the
blocks of A and B whose K index lies in its range, computes the partial product
C~_i = op(A_i) op(B_i) with the library's own plan and execute, and the C~_i are summed
into C.  The norm filter acts on single block products, so splitting K keeps exactly
the products the undivided multiply keeps, and the union of the partial patterns is
the undivided C pattern.

The sum is a reduce-scatter in a fixed order:
  1. the partial patterns (block rows and columns, CSR order) are gathered on every
     process and merged into the union pattern;
  2. the union's blocks are cut into P contiguous ranges of about equal element counts,
     range q owned by process q;
  3. one all-to-all moves, from every process, the run of its partial product that falls
     in each owner's range (a contiguous run: each partial keeps CSR order);
  4. each owner adds its received parts with bst_sum_parts, part 0 first, so the bits do
     not depend on the process count's layout or on the transport.
Each process sends and receives about S_C elements in step 3, as in the paper's
reduction.  C_in (times beta) enters once, through process 0's partial product.

Host functions (k_ranges, select_k_range, exchange_layout) are plain numpy and hold no
arithmetic of the product; gather_patterns and exchange run over torch.distributed (NCCL
between GPUs, gloo for CPU tensors); multiply_ksplit runs the whole step on the GPU."""
from dataclasses import dataclass

import numpy as np

__all__ = ["k_index", "k_ranges", "select_k_range", "Layout", "exchange_layout",
           "gather_patterns", "exchange", "multiply_ksplit", "KSplitResult",
           "select_tensor_range", "tensor_fold", "tensor_unfold", "result_block_sizes",
           "contract_ksplit"]


def k_index(rows, cols, trans, side):
    """The K block index of every stored block of A (side "A") or B (side "B"):
    op(A) = A has K along its block columns, A^T along its block rows; op(B) = B along
    its block rows, B^T along its block columns."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    if side == "A":
        return cols if trans == "N" else rows
    if side == "B":
        return rows if trans == "N" else cols
    raise ValueError("side must be 'A' or 'B'")


def k_ranges(ka, a_elems, kb, b_elems, k_sizes, world):
    """Boundaries r[0] = 0 <= ... <= r[world] = K of contiguous K-block ranges of about
    equal work.  The work of K block k is bounded by (elements of the op(A) blocks in
    k) x (elements of the op(B) blocks in k) / k_size[k]: the multiply-adds of all its
    products before the filter."""
    k_sizes = np.asarray(k_sizes, np.float64)
    K = len(k_sizes)
    wa = np.bincount(np.asarray(ka, np.int64), weights=np.asarray(a_elems, np.float64),
                     minlength=K)
    wb = np.bincount(np.asarray(kb, np.int64), weights=np.asarray(b_elems, np.float64),
                     minlength=K)
    w = wa * wb / np.maximum(k_sizes, 1.0)
    cum = np.concatenate(([0.0], np.cumsum(w)))
    total = cum[-1]
    r = np.zeros(world + 1, np.int64)
    for q in range(1, world):
        r[q] = np.searchsorted(cum, total * q / world, side="left")
    r[world] = K
    return np.maximum.accumulate(np.clip(r, 0, K))


def select_k_range(row_sizes, col_sizes, rows, cols, data, trans, side, lo, hi):
    """The blocks of a host block-sparse matrix (CSR order, blocks packed in that order)
    whose K index lies in [lo, hi): (rows, cols, data), same block-index space."""
    rows = np.asarray(rows, np.int32)
    cols = np.asarray(cols, np.int32)
    lens = (np.asarray(row_sizes, np.int64)[rows] * np.asarray(col_sizes, np.int64)[cols])
    k = k_index(rows, cols, trans, side)
    keep = (k >= lo) & (k < hi)
    return rows[keep], cols[keep], np.asarray(data, np.float64)[np.repeat(keep, lens)]


@dataclass
class Layout:
    """Where every block of every partial product goes (identical on every process).

    rows, cols, offsets: the union C pattern in CSR order, offsets[nblocks] elements;
    owner[q] .. owner[q+1]: the union blocks process q owns;
    send[i][q]: elements of process i's partial product that go to process q (a
    contiguous run of it, runs in increasing q);
    src_off[q]: int64[P, nblocks owned by q], the offset of each owned block's elements
    in q's receive buffer (the runs from processes 0 .. P-1 one after another), -1 where
    that process's partial product has no such block."""
    rows: np.ndarray
    cols: np.ndarray
    offsets: np.ndarray
    owner: np.ndarray
    send: np.ndarray
    src_off: list

    def owned(self, q):
        """(rows, cols, offsets from 0) of the blocks process q owns."""
        a, b = int(self.owner[q]), int(self.owner[q + 1])
        return self.rows[a:b], self.cols[a:b], self.offsets[a:b + 1] - self.offsets[a]


def exchange_layout(patterns, row_sizes, col_sizes):
    """The Layout of P partial products given their patterns [(rows, cols), ...] (each in
    CSR order: rows non-decreasing, columns increasing inside a row) and the block sizes
    of C's rows and columns."""
    P = len(patterns)
    rs = np.asarray(row_sizes, np.int64)
    cs = np.asarray(col_sizes, np.int64)
    ncol = max(len(cs), 1)
    keys = []
    for r, c in patterns:
        k = np.asarray(r, np.int64) * ncol + np.asarray(c, np.int64)
        if len(k) > 1 and not (np.diff(k) > 0).all():
            raise ValueError("a partial pattern is not in CSR order")
        keys.append(k)
    ukey = np.unique(np.concatenate(keys)) if keys else np.zeros(0, np.int64)
    urows = (ukey // ncol).astype(np.int32)
    ucols = (ukey % ncol).astype(np.int32)
    ulen = rs[urows] * cs[ucols]
    uoff = np.concatenate(([0], np.cumsum(ulen))).astype(np.int64)
    nU = len(ukey)
    # owners: contiguous block ranges of about equal element counts
    owner = np.zeros(P + 1, np.int64)
    for q in range(1, P):
        owner[q] = np.searchsorted(uoff[:-1], uoff[-1] * q / P, side="left") if nU else 0
    owner[P] = nU
    owner = np.maximum.accumulate(np.clip(owner, 0, nU))
    # each partial's blocks as union indices, their element offsets, and its runs
    send = np.zeros((P, P), np.int64)
    where, loffs, cuts = [], [], []
    for i in range(P):
        ui = np.searchsorted(ukey, keys[i])
        loff = np.concatenate(([0], np.cumsum(ulen[ui]))).astype(np.int64)
        cut = np.searchsorted(ui, owner)  # local blocks [cut[q], cut[q+1]) go to q
        send[i] = loff[cut[1:]] - loff[cut[:-1]]
        where.append(ui)
        loffs.append(loff)
        cuts.append(cut)
    src_off = []
    for q in range(P):
        a, b = int(owner[q]), int(owner[q + 1])
        tab = np.full((P, b - a), -1, np.int64)
        base = 0
        for i in range(P):
            j0, j1 = int(cuts[i][q]), int(cuts[i][q + 1])
            if j1 > j0:
                tab[i, where[i][j0:j1] - a] = base + loffs[i][j0:j1] - loffs[i][j0]
            base += int(send[i, q])
        src_off.append(tab)
    return Layout(urows, ucols, uoff, owner, send, src_off)


def gather_patterns(rows, cols, group=None, device="cpu"):
    """Every process's (rows, cols) on every process (all_gather of the counts, then of
    the patterns padded to the largest)."""
    import torch
    import torch.distributed as dist
    P = dist.get_world_size(group)
    n = torch.tensor([len(rows)], dtype=torch.int64, device=device)
    ns = [torch.zeros_like(n) for _ in range(P)]
    dist.all_gather(ns, n, group=group)
    ns = [int(x.item()) for x in ns]
    mx = max(max(ns), 1)
    mine = torch.full((2, mx), -1, dtype=torch.int64, device=device)
    if len(rows):
        mine[0, :len(rows)] = torch.as_tensor(np.asarray(rows, np.int64), device=device)
        mine[1, :len(cols)] = torch.as_tensor(np.asarray(cols, np.int64), device=device)
    allp = [torch.empty_like(mine) for _ in range(P)]
    dist.all_gather(allp, mine, group=group)
    out = []
    for q in range(P):
        a = allp[q].cpu().numpy()
        out.append((a[0, :ns[q]].astype(np.int32), a[1, :ns[q]].astype(np.int32)))
    return out


def exchange(part, layout, group=None):
    """This process's receive buffer: the runs of every process's partial product that
    fall in its owned range, process 0's first (one all_to_all_single over `group`).
    `part` is this process's packed partial product (a 1-D FP64 tensor)."""
    import torch
    import torch.distributed as dist
    q = dist.get_rank(group)
    P = dist.get_world_size(group)
    send = [int(x) for x in layout.send[q]]
    recv = [int(layout.send[i, q]) for i in range(P)]
    out = torch.empty(sum(recv), dtype=part.dtype, device=part.device)
    dist.all_to_all_single(out, part[:sum(send)], output_split_sizes=recv,
                           input_split_sizes=send, group=group)
    return out


@dataclass
class KSplitResult:
    """The blocks of C this process owns (rows, cols, element offsets from 0, device
    data), the layout they come from and the local plan of the partial product."""
    rows: np.ndarray
    cols: np.ndarray
    offsets: np.ndarray
    data: object
    layout: Layout
    plan: object
    _tables: tuple = ()


def sum_owned(layout, q, recv, device=0, stream=None):
    """Process q's owned blocks of C: its receive buffer summed by bst_sum_parts on the
    GPU.  Returns (rows, cols, offsets, data, tables); `tables` are the device copies of
    the layout the queued kernel reads (keep them until it has run)."""
    import torch

    from . import bst
    rows, cols, offs = layout.owned(q)
    n = len(rows)
    dev = torch.device("cuda", device)
    dst = torch.empty(int(offs[-1]), dtype=torch.float64, device=dev)
    tables = ()
    if n:
        d_off = torch.as_tensor(np.ascontiguousarray(offs, np.int64)).to(dev)
        s_off = torch.as_tensor(np.ascontiguousarray(layout.src_off[q], np.int64)).to(dev)
        bst.bst_sum_parts(bst.context(device), len(layout.owner) - 1, n, d_off, s_off,
                          recv, dst, stream)
        tables = (d_off, s_off, recv)
    return rows, cols, offs, dst, tables


def multiply_ksplit(A, B, row_sizes, col_sizes, C_in=None, alpha=1.0, beta=0.0, eps=0.0,
                    transa="N", transb="N", precision=None, group=None, device=0):
    """C = alpha op(A) op(B) + beta C_in over the processes of `group`, K divided among
    them: A and B (library matrices on this process's GPU) hold this process's blocks
    of the K range it was given (select_k_range cuts them from whole host matrices);
    row_sizes and col_sizes are C's block sizes (op(A)'s rows, op(B)'s columns); C_in
    is used on process 0 only.  Returns this process's owned part of C.  Every process
    of the group must call it (collectives)."""
    import torch.distributed as dist

    from . import bst
    if precision is None:
        precision = bst.BST_FP64
    q = dist.get_rank(group)
    plan = bst.multiply_plan(A, B, C_in if q == 0 else None, eps, transa, transb, device)
    C = plan.alloc_result(device)
    plan.execute(alpha, beta if q == 0 else 0.0, precision)
    rows, cols, _ = C.index()
    nloc = C.info[3]  # elements of the partial product
    pdev = f"cuda:{device}" if dist.get_backend(group) == "nccl" else "cpu"
    layout = exchange_layout(gather_patterns(rows, cols, group, pdev), row_sizes, col_sizes)
    part = C.data[:nloc]
    if pdev == "cpu":  # a host transport: the runs travel through host memory
        part = part.cpu()
    recv = exchange(part, layout, group).to(C.data.device)
    r, c, o, data, tables = sum_owned(layout, q, recv, device)
    return KSplitResult(r, c, o, data, layout, plan, tables)


# ---- contractions -------------------------------------------------------------------
#
# The same split for a tensor contraction whose contracted index is long (paper Sec. 4:
# three-centre integrals T(P, mu, nu), P the auxiliary index, contracted with U(P, nu,
# lam)): each process holds the blocks of T1 and T2 whose index along a contracted mode
# pair lies in its range, contracts them with the library, and the partial results R~_i
# are summed as above, R's blocks seen as the rows and columns of its fold (all modes
# but the last as rows, the last as columns: R's canonical block order is then CSR
# order, and a block's elements are the row-major fold of its own).


def select_tensor_range(block_sizes, index, data, mode, lo, hi):
    """The blocks of a host tensor (canonical order, blocks packed in that order) whose
    index along `mode` lies in [lo, hi): (index, data)."""
    index = np.asarray(index, np.int32)
    lens = np.ones(len(index), np.int64)
    for d, s in enumerate(block_sizes):
        lens *= np.asarray(s, np.int64)[index[:, d]]
    keep = (index[:, mode] >= lo) & (index[:, mode] < hi)
    return index[keep], np.asarray(data, np.float64)[np.repeat(keep, lens)]


def tensor_fold(index, block_sizes):
    """A tensor's blocks as (rows, cols) of its fold -- rows = the modes but the last
    (mixed radix, mode 0 slowest), cols = the last mode -- with the fold's row and column
    block sizes."""
    index = np.asarray(index, np.int64).reshape(len(index), -1)
    rank = index.shape[1]
    sizes = [np.asarray(s, np.int64) for s in block_sizes]
    if rank == 1:
        return (np.zeros(len(index), np.int32), index[:, 0].astype(np.int32),
                np.ones(1, np.int64), sizes[0])
    rows = np.zeros(len(index), np.int64)
    row_sizes = np.ones(1, np.int64)
    for d in range(rank - 1):
        rows = rows * len(sizes[d]) + index[:, d]
        row_sizes = np.outer(row_sizes, sizes[d]).reshape(-1)
    return rows.astype(np.int32), index[:, -1].astype(np.int32), row_sizes, sizes[-1]


def tensor_unfold(rows, cols, block_sizes):
    """The block index tuples (nblocks x rank) of fold rows and columns."""
    nblk = [len(s) for s in block_sizes]
    rank = len(nblk)
    out = np.zeros((len(rows), rank), np.int32)
    out[:, -1] = cols
    r = np.asarray(rows, np.int64).copy()
    for d in range(rank - 2, -1, -1):
        out[:, d] = r % nblk[d]
        r //= nblk[d]
    return out


def result_block_sizes(sizes1, sizes2, f1, f2, result_order=None):
    """Per-mode block sizes of a contraction's result: the free modes (f1..., f2...),
    result mode r being free slot result_order[r]."""
    free = [sizes1[d] for d in f1] + [sizes2[d] for d in f2]
    order = range(len(free)) if result_order is None else result_order
    return [np.asarray(free[r], np.int64) for r in order]


def contract_ksplit(T1, T2, c1, c2, f1, f2, r_block_sizes, result_order=None, R_in=None,
                    alpha=1.0, beta=0.0, eps=0.0, precision=None, group=None, device=0):
    """R = alpha sum T1 T2 + beta R_in over the processes of `group`, a contracted mode
    pair divided among them: T1 and T2 (library tensors on this process's GPU) hold this
    process's blocks of it (select_tensor_range cuts them from whole host tensors), R_in
    is used on process 0 only; r_block_sizes are R's per-mode block sizes
    (result_block_sizes).  Returns this process's owned blocks of R as a KSplitResult
    whose rows and columns are those of R's fold (tensor_unfold gives the index tuples).
    Every process of the group must call it."""
    import torch.distributed as dist

    from . import bst
    if precision is None:
        precision = bst.BST_FP64
    q = dist.get_rank(group)
    plan = bst.contract(T1, T2, c1, c2, f1, f2, result_order, R_in if q == 0 else None,
                        alpha, beta if q == 0 else 0.0, eps, precision, 1, device)
    R = plan.result
    idx, _ = R.index()
    rows, cols, row_sizes, col_sizes = tensor_fold(idx, r_block_sizes)
    nloc = R.info[2]
    pdev = f"cuda:{device}" if dist.get_backend(group) == "nccl" else "cpu"
    layout = exchange_layout(gather_patterns(rows, cols, group, pdev), row_sizes, col_sizes)
    part = R.data[:nloc]
    if pdev == "cpu":
        part = part.cpu()
    recv = exchange(part, layout, group).to(R.data.device)
    r, c, o, data, tables = sum_owned(layout, q, recv, device)
    return KSplitResult(r, c, o, data, layout, plan, tables)
