"""Full-size workloads compared WHOLE against the CPU oracle: every C block index and
element offset and every stack array bit for bit, and all of C within the tolerance of
its arithmetic (native FP64 1e-12, emulated FP64 1e-11 relative Frobenius).

* banded 4000 x 4000 blocks of sizes 5/13/23, eps = 1e-8 (2.1e10 flop; the oracle takes
  about 20 s on one core);
* tall-skinny A^T B, 100000 x 400 blocks (2.4e9 flop), unsplit, split-K 4 and auto;
* the rank-3 contraction R(mu, lam) = T(P, mu, nu) U(P, nu, lam) through the autograd
  wrapper: R whole against the oracle, loss = 1/2 ||R||^2, loss.backward() against the
  oracle's adjoint (on seeded block subsets), central differences on 50 entries.
"""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, run_multiply, to_lib
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import BSTensor, banded, rank3, tall_skinny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _assert_exact(got, ref):
    assert (got["rows"] == ref["rows"]).all() and (got["cols"] == ref["cols"]).all()
    assert (got["offsets"] == ref["offsets"]).all()
    st = got["stats"]
    assert st["n_candidates"] == ref["ncandidates"]
    assert st["n_filtered"] == ref["nfiltered"]
    assert st["n_stack"] == len(ref["a_off"])
    assert st["flops"] == ref["flops"]
    for k in ("mnk", "bucket_ptr", "a_off", "b_off", "c_off"):
        assert got[k].shape == ref[k].shape and (got[k] == ref[k]).all(), k


def _per_block_rel(data, ref, offs, lens):
    """Largest relative Frobenius error over the C blocks (each block against itself)."""
    d = (np.asarray(data) - ref) ** 2
    r = ref ** 2
    cs = np.concatenate([[0.0], np.cumsum(d)])
    cr = np.concatenate([[0.0], np.cumsum(r)])
    e = np.sqrt(cs[offs + lens] - cs[offs])
    n = np.sqrt(cr[offs + lens] - cr[offs])
    ok = n > 0
    return float((e[ok] / n[ok]).max()) if ok.any() else 0.0


def test_banded_full_size_exact():
    import torch
    p = banded()
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    got = run_multiply(p, stacks=True)
    _assert_exact(got, ref)
    assert 0 < ref["nfiltered"] < ref["ncandidates"]
    assert rel_fro(got["data"], ref["data"]) <= 1e-12
    # emulated FP64 on the same plan, whole C within 1e-11: the first emulated execute
    # runs the C-block kernel, the second the tcgen05 panel kernel (default policy)
    plan = got["plan"]
    ne = plan.result.info[3]
    for panel in (False, True):
        assert bst.bst_plan_emu_costs(plan.handle)["panel"] == panel
        plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
        emu = plan.result.data[:ne].cpu().numpy()
        assert rel_fro(emu, ref["data"]) <= 1e-11, panel
    plan.stats()  # reports a timeout of the panel kernel, if any


def test_tall_skinny_full_size_exact():
    import torch
    p = tall_skinny()
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps, p.transa, p.transb)
    got = run_multiply(p, stacks=True)
    _assert_exact(got, ref)
    assert rel_fro(got["data"], ref["data"]) <= 1e-12
    plan = got["plan"]
    ne = plan.result.info[3]
    for split in (4, 0):
        plan.execute(1.0, 0.0, bst.BST_FP64, split)
        torch.cuda.synchronize()
        assert rel_fro(plan.result.data[:ne].cpu().numpy(), ref["data"]) <= 1e-12
    plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
    torch.cuda.synchronize()
    assert rel_fro(plan.result.data[:ne].cpu().numpy(), ref["data"]) <= 1e-11


def _subset(t, sel):
    """The blocks `sel` (sorted) of a block-sparse tensor, with their data."""
    offs, lens = t.offsets, t.block_lens
    idx = np.concatenate([np.arange(offs[b], offs[b] + lens[b]) for b in sel])
    return BSTensor(t.block_sizes, t.index[sel], t.data[idx]), idx


def _gather_blocks(full_index, full_offsets, full_lens, data, want_index):
    """Data of the blocks `want_index` (rows of block tuples) out of a packed tensor."""
    pos = {tuple(r): q for q, r in enumerate(full_index.tolist())}
    q = np.array([pos[tuple(r)] for r in want_index.tolist()], np.int64)
    return np.concatenate([data[full_offsets[b]:full_offsets[b] + full_lens[b]] for b in q])


def test_rank3_full_size_autograd_exact():
    """Forward R whole against the oracle; loss = 1/2 ||R||^2 and loss.backward() through
    the autograd wrapper; T.grad and U.grad against the oracle's adjoint on 1/16 of the
    blocks of each (seeded; a gradient block depends only on its own block, the other
    operand and dR, so the oracle computes it exactly from the subset); central
    differences on 50 entries through the wrapper."""
    import torch
    from paper_1910_13555_gb300 import autograd
    w = rank3()
    args = (w.c1, w.c2, w.f1, w.f2, w.result_order)
    t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data)
    t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data)
    t1.data.requires_grad_(True)
    t2.data.requires_grad_(True)
    r, plan = autograd.contract(t1, t2, *args)
    loss = 0.5 * (r * r).sum()
    loss.backward()
    torch.cuda.synchronize()
    # forward: the whole result against the oracle
    ref = oracle.contract(w.T1, w.T2, *args)
    idx, offs = bst.bst_tensor_get_index(bst.bst_plan_result_tensor(plan.handle))
    assert (idx == ref["index"]).all() and (offs == ref["offsets"]).all()
    R = r.detach()[:len(ref["data"])].cpu().numpy()
    assert rel_fro(R, ref["data"]) <= 1e-12
    rlens = np.diff(np.r_[ref["offsets"], len(ref["data"])])
    # backward: dR = R; the oracle's adjoint on a seeded 1/16 of T's and of U's blocks
    rng = np.random.default_rng(5)
    g1, g2 = t1.data.grad.cpu().numpy(), t2.data.grad.cpu().numpy()
    for side in (0, 1):
        full = (w.T1, w.T2)[side]
        sel = np.sort(rng.choice(full.nblocks, full.nblocks // 16, replace=False))
        sub, eidx = _subset(full, sel)
        T1s, T2s = (sub, w.T2) if side == 0 else (w.T1, sub)
        rs = oracle.contract(T1s, T2s, *args)
        dR = _gather_blocks(ref["index"], ref["offsets"], rlens, ref["data"], rs["index"])
        d = oracle.contract_adjoint(T1s, T2s, *args, None, 1.0, 0.0, 0.0, dR)[side]
        assert rel_fro((g1, g2)[side][eidx], d) <= 1e-12, side
    # central differences on 25 entries of T and 25 of U, each loss through the wrapper
    # (the loss is quadratic in every entry: no truncation error)
    h = 1e-6
    L = float(loss.detach())
    with torch.no_grad():
        for M, g in ((t1, t1.data.grad), (t2, t2.data.grad)):
            for e in rng.choice(M.data.numel(), 25, replace=False):
                old = float(M.data[e])
                vals = []
                for x in (old + h, old - h):
                    M.data[e] = x
                    rr = autograd.BlockSparseContractFn.apply(t1.data, t2.data, None, plan, 1.0,
                                                              0.0, bst.BST_FP64)
                    vals.append(0.5 * float((rr * rr).sum()))
                M.data[e] = old
                fd = (vals[0] - vals[1]) / (2 * h)
                gv = float(g[e])
                assert abs(fd - gv) <= 1e-7 * max(1.0, abs(gv)) + 8 * 2.0 ** -52 * L / h
