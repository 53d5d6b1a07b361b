"""The K-split product on the GPU (paper Sec. 3.1): bst_sum_parts against the fixed-order
sum written out in numpy (bit-exact), and the whole split -- partial products by the
library's multiply, the exchange layout, the owners' sums by bst_sum_parts -- against
the CPU oracle's undivided product.  Processes are simulated one after another on one
GPU (each owner's receive buffer assembled from the partial products as the all-to-all
would deliver it); multiply_ksplit itself runs in a one-process group, over NCCL and
over gloo."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_util import require_gpu
from paper_1910_13555_gb300 import bst, ksplit
from paper_1910_13555_gb300.workloads import BSMatrix, tall_skinny

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _np_fixed_sum(nblocks, dst_off, src_off, src, nparts):
    out = np.zeros(int(dst_off[-1]))
    for u in range(nblocks):
        n = int(dst_off[u + 1] - dst_off[u])
        acc = None
        for i in range(nparts):
            o = int(src_off[i * nblocks + u])
            if o >= 0:
                acc = src[o:o + n].copy() if acc is None else acc + src[o:o + n]
        if acc is not None:
            out[dst_off[u]:dst_off[u] + n] = acc
    return out


@pytest.mark.parametrize("nparts", [1, 2, 4, 7])
def test_sum_parts_bit_exact_fixed_order(nparts):
    import torch
    rng = np.random.default_rng(nparts)
    nb = 3001  # several CTAs, a ragged tail
    lens = rng.integers(1, 600, nb)
    dst_off = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
    src_off = np.full(nparts * nb, -1, np.int64)
    pos = 0
    for i in range(nparts):
        for u in range(nb):
            if rng.random() < 0.7 or (i == 0 and u % 97 == 0):
                src_off[i * nb + u] = pos
                pos += int(lens[u])
    src_off[::nparts * 13 + 1] = -1  # some blocks no part has (written as 0)
    src = rng.standard_normal(max(pos, 1)) * 10.0 ** rng.integers(-8, 8, max(pos, 1))
    dev = torch.device("cuda", 0)
    d = torch.full((int(dst_off[-1]),), np.nan, dtype=torch.float64, device=dev)
    t_dst, t_src = torch.as_tensor(dst_off).to(dev), torch.as_tensor(src_off).to(dev)
    t_in = torch.as_tensor(src).to(dev)
    bst.bst_sum_parts(bst.context(0), nparts, nb, t_dst, t_src, t_in, d)
    torch.cuda.synchronize()
    ref = _np_fixed_sum(nb, dst_off, src_off, src, nparts)
    assert np.array_equal(d.cpu().numpy(), ref)
    bst.bst_sum_parts(bst.context(0), nparts, 0, t_dst, t_src, t_in, d)  # nothing to do
    with pytest.raises(bst.BstError) as e:
        bst.bst_sum_parts(bst.context(0), 0, nb, t_dst, t_src, t_in, d)
    assert e.value.name == "BST_ERR_INVALID_ARG"


def _problem(eps):
    return tall_skinny(seed=21, nk=20000, nmn=120, window=20, p=0.2, eps=eps)


def _cut(M, trans, side, lo, hi):
    r, c, d = ksplit.select_k_range(M.row_sizes, M.col_sizes, M.rows, M.cols, M.data, trans,
                                    side, lo, hi)
    return BSMatrix(M.row_sizes, M.col_sizes, r, c, d)


@pytest.mark.parametrize("P", [2, 3, 8])
def test_simulated_ksplit_against_oracle(P):
    import torch
    p = _problem(eps=30.0)
    full = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb)
    assert full["nfiltered"] > 0
    A, B = p.A, p.B
    ka = ksplit.k_index(A.rows, A.cols, "T", "A")
    kb = ksplit.k_index(B.rows, B.cols, "N", "B")
    ea = A.row_sizes[A.rows].astype(np.int64) * A.col_sizes[A.cols]
    eb = B.row_sizes[B.rows].astype(np.int64) * B.col_sizes[B.cols]
    r = ksplit.k_ranges(ka, ea, kb, eb, A.row_sizes, P)
    mk = lambda m: bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)
    parts, pats, keep = [], [], []
    for i in range(P):
        Ai, Bi = mk(_cut(A, "T", "A", r[i], r[i + 1])), mk(_cut(B, "N", "B", r[i], r[i + 1]))
        plan = bst.multiply(Ai, Bi, None, 1.0, 0.0, p.eps, "T", "N")
        rows, cols, _ = plan.result.index()
        pats.append((rows, cols))
        parts.append(plan.result.data[:plan.result.info[3]])
        keep.append((plan, Ai, Bi))
    lay = ksplit.exchange_layout(pats, A.col_sizes, B.col_sizes)
    assert np.array_equal(lay.rows, full["rows"]) and np.array_equal(lay.cols, full["cols"])
    out, host = [], [x.cpu().numpy() for x in parts]
    for q in range(P):
        chunks = []
        for i in range(P):
            s0 = int(lay.send[i, :q].sum())
            chunks.append(parts[i][s0:s0 + int(lay.send[i, q])])
        recv = torch.cat(chunks)
        _, _, offs, data, tables = ksplit.sum_owned(lay, q, recv)
        torch.cuda.synchronize()
        got = data.cpu().numpy()
        ref = _np_fixed_sum(len(offs) - 1, offs, lay.src_off[q].reshape(-1), recv.cpu().numpy(), P)
        assert np.array_equal(got, ref)  # the fixed order, bit for bit
        out.append(got)
    got = np.concatenate(out)
    rel = np.linalg.norm(got - full["data"]) / np.linalg.norm(full["data"])
    assert rel <= 1e-12
    assert sum(h.size for h in host) == lay.send.sum()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np, torch, torch.distributed as dist
import oracle
import test_gpu_ksplit as T
from paper_1910_13555_gb300 import bst, ksplit
backend = os.environ["BACKEND"]
torch.cuda.set_device(0)
dist.init_process_group(backend, rank=0, world_size=1,
                        init_method="tcp://127.0.0.1:" + os.environ["PORT"])
p = T._problem(eps=30.0)
mk = lambda m: bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)
res = ksplit.multiply_ksplit(mk(p.A), mk(p.B), p.A.col_sizes, p.B.col_sizes, eps=p.eps,
                             alpha=0.5, transa="T", transb="N")
torch.cuda.synchronize()
full = oracle.multiply(p.A, p.B, None, 0.5, 0.0, p.eps, "T", "N")
assert np.array_equal(res.rows, full["rows"]) and np.array_equal(res.cols, full["cols"])
got = res.data.cpu().numpy()
rel = np.linalg.norm(got - full["data"]) / np.linalg.norm(full["data"])
assert rel <= 1e-12, rel
dist.destroy_process_group()
print("ok", rel)
"""


@pytest.mark.parametrize("backend", ["nccl", "gloo"])
def test_multiply_ksplit_one_process_group(backend):
    env = dict(os.environ, BACKEND=backend, PORT=str(_free_port()), NCCL_NVLS_ENABLE="0")
    pr = subprocess.run([sys.executable, "-c", _WORKER.format(root=ROOT)], env=env, cwd=ROOT,
                        capture_output=True, text=True, timeout=300)
    assert pr.returncode == 0, pr.stderr[-3000:]
    # the communication libraries print their own lines too
    assert any(line.startswith("ok ") for line in pr.stdout.splitlines()), pr.stdout


def test_simulated_ksplit_with_cin_alpha_beta():
    """alpha on every partial product, beta C_in on process 0's only (C_in has blocks no
    product reaches), 3 processes simulated on one GPU, against the undivided oracle."""
    import torch
    rng = np.random.default_rng(22)
    p = _problem(eps=30.0)
    A, B = p.A, p.B
    rs, cs = A.col_sizes, B.col_sizes
    full0 = oracle.multiply(A, B, None, 1.0, 0.0, p.eps, "T", "N")
    keep = rng.random(len(full0["rows"])) < 0.3
    pairs = sorted(set(zip(full0["rows"][keep].tolist(), full0["cols"][keep].tolist())) |
                   set(zip(rng.integers(0, len(rs), 25).tolist(),
                           rng.integers(0, len(cs), 25).tolist())))
    ci_r = np.array([a for a, _ in pairs], np.int32)
    ci_c = np.array([b for _, b in pairs], np.int32)
    ci_d = rng.uniform(-1, 1, int((rs[ci_r].astype(np.int64) * cs[ci_c]).sum()))
    Ci = BSMatrix(rs, cs, ci_r, ci_c, ci_d)
    alpha, beta = -0.75, 1.5
    full = oracle.multiply(A, B, Ci, alpha, beta, p.eps, "T", "N")
    ka = ksplit.k_index(A.rows, A.cols, "T", "A")
    kb = ksplit.k_index(B.rows, B.cols, "N", "B")
    ea = A.row_sizes[A.rows].astype(np.int64) * A.col_sizes[A.cols]
    eb = B.row_sizes[B.rows].astype(np.int64) * B.col_sizes[B.cols]
    P = 3
    r = ksplit.k_ranges(ka, ea, kb, eb, A.row_sizes, P)
    mk = lambda m: bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)
    parts, pats, keep_alive = [], [], []
    for i in range(P):
        Ai, Bi = mk(_cut(A, "T", "A", r[i], r[i + 1])), mk(_cut(B, "N", "B", r[i], r[i + 1]))
        Cii = mk(Ci) if i == 0 else None
        plan = bst.multiply(Ai, Bi, Cii, alpha, beta if i == 0 else 0.0, p.eps, "T", "N")
        rows, cols, _ = plan.result.index()
        pats.append((rows, cols))
        parts.append(plan.result.data[:plan.result.info[3]])
        keep_alive.append((plan, Ai, Bi, Cii))
    lay = ksplit.exchange_layout(pats, rs, cs)
    assert np.array_equal(lay.rows, full["rows"]) and np.array_equal(lay.cols, full["cols"])
    out = []
    for q in range(P):
        recv = torch.cat([parts[i][int(lay.send[i, :q].sum()):int(lay.send[i, :q + 1].sum())]
                          for i in range(P)])
        _, _, _, data, _ = ksplit.sum_owned(lay, q, recv)
        torch.cuda.synchronize()
        out.append(data.cpu().numpy())
    got = np.concatenate(out)
    assert np.linalg.norm(got - full["data"]) / np.linalg.norm(full["data"]) <= 1e-12


def _rank3_small():
    from paper_1910_13555_gb300.workloads import rank3
    return rank3(nP=300, sP=12, nao=60, window=8, p=0.3)


def test_simulated_contraction_split_against_oracle():
    """The rank-3 contraction split over P among 3 processes simulated on one GPU: the
    library's partial contractions, the fold layout and bst_sum_parts, against the
    oracle's undivided contraction."""
    import torch
    from paper_1910_13555_gb300.workloads import BSTensor
    w = _rank3_small()
    full = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order)
    rsz = ksplit.result_block_sizes(w.T1.block_sizes, w.T2.block_sizes, w.f1, w.f2,
                                    w.result_order)
    nP = len(w.T1.block_sizes[0])
    bounds = [0, nP // 3, 2 * nP // 3, nP]
    parts, pats, keep = [], [], []
    for i in range(3):
        i1, d1 = ksplit.select_tensor_range(w.T1.block_sizes, w.T1.index, w.T1.data,
                                            w.c1[0], bounds[i], bounds[i + 1])
        i2, d2 = ksplit.select_tensor_range(w.T2.block_sizes, w.T2.index, w.T2.data,
                                            w.c2[0], bounds[i], bounds[i + 1])
        t1 = bst.Tensor.from_host(w.T1.block_sizes, i1, d1)
        t2 = bst.Tensor.from_host(w.T2.block_sizes, i2, d2)
        plan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order)
        idx, _ = plan.result.index()
        rows, cols, row_sizes, col_sizes = ksplit.tensor_fold(idx, rsz)
        pats.append((rows, cols))
        parts.append(plan.result.data[:plan.result.info[2]])
        keep.append((plan, t1, t2))
    lay = ksplit.exchange_layout(pats, row_sizes, col_sizes)
    assert np.array_equal(ksplit.tensor_unfold(lay.rows, lay.cols, rsz), full["index"])
    out = []
    for q in range(3):
        recv = torch.cat([parts[i][int(lay.send[i, :q].sum()):int(lay.send[i, :q + 1].sum())]
                          for i in range(3)])
        _, _, _, data, _ = ksplit.sum_owned(lay, q, recv)
        torch.cuda.synchronize()
        out.append(data.cpu().numpy())
    got = np.concatenate(out)
    assert np.linalg.norm(got - full["data"]) / np.linalg.norm(full["data"]) <= 1e-12


_CWORKER = r"""
import os, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np, torch, torch.distributed as dist
import oracle
import test_gpu_ksplit as T
from paper_1910_13555_gb300 import bst, ksplit
torch.cuda.set_device(0)
dist.init_process_group("nccl", rank=0, world_size=1,
                        init_method="tcp://127.0.0.1:" + os.environ["PORT"])
w = T._rank3_small()
t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data)
t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data)
rsz = ksplit.result_block_sizes(w.T1.block_sizes, w.T2.block_sizes, w.f1, w.f2, w.result_order)
res = ksplit.contract_ksplit(t1, t2, w.c1, w.c2, w.f1, w.f2, rsz, w.result_order, alpha=2.0)
torch.cuda.synchronize()
full = oracle.contract(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order, alpha=2.0)
assert np.array_equal(ksplit.tensor_unfold(res.rows, res.cols, rsz), full["index"])
got = res.data.cpu().numpy()
rel = np.linalg.norm(got - full["data"]) / np.linalg.norm(full["data"])
assert rel <= 1e-12, rel
dist.destroy_process_group()
print("ok", rel)
"""


def test_contract_ksplit_one_process_group():
    env = dict(os.environ, PORT=str(_free_port()), NCCL_NVLS_ENABLE="0")
    pr = subprocess.run([sys.executable, "-c", _CWORKER.format(root=ROOT)], env=env, cwd=ROOT,
                        capture_output=True, text=True, timeout=300)
    assert pr.returncode == 0, pr.stderr[-3000:]
    assert any(line.startswith("ok ") for line in pr.stdout.splitlines()), pr.stdout
