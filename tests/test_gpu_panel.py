"""Emulated FP64 on the tcgen05 panel kernel (per inner block k: the op(A) blocks of
block column k times the op(B) blocks of block row k as one dense tensor-core product),
against the CPU oracle through the C ABI.

Values within 1e-11 relative Frobenius error over all of C and, with block scales that
span eight decades, within 1e-11 on every C block; integer-valued inputs bit-exact;
patterns bit-exact; repeat executes bitwise equal (the slot sums are integer, in a
fixed order); transposes, alpha, beta with C_in (including C_in blocks that no product
reaches), the filter, and a plan the kernel does not take (blocks above its tiles)."""
import contextlib

import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from helpers import random_matrix, transpose_matrix
from paper_1910_13555_gb300 import bst
from paper_1910_13555_gb300.workloads import BSMatrix, Problem, banded, batched

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@contextlib.contextmanager
def panel_mode(mode):
    ctx = bst.context()
    old = bst.bst_tune_get(ctx, bst.BST_TUNE_EMU_PANEL)
    bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_PANEL, mode)
    try:
        yield
    finally:
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_PANEL, old)


def run_emu(p, mode=2):
    import torch
    with panel_mode(mode):
        A, B = to_lib(p.A), to_lib(p.B)
        Ci = to_lib(p.C_in) if p.C_in is not None else None
        plan = bst.multiply_plan(A, B, Ci, p.eps, p.transa, p.transb)
        C = plan.alloc_result()
        C.data.fill_(float("nan"))
        plan.execute(p.alpha, p.beta, bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
        costs = bst.bst_plan_emu_costs(plan.handle)
        st = plan.stats()  # reports a device-side timeout of the panel kernel, if any
        rows, cols, offs = C.index()
        n = C.info[3]
        out = dict(rows=rows, cols=cols, offsets=offs, data=C.data[:n].cpu().numpy(),
                   costs=costs, stats=st, plan=plan, mats=(A, B, Ci), C=C)
    return out


def check(p, mode=2, tol=TOL, expect_panel=True):
    ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, p.transa, p.transb)
    got = run_emu(p, mode)
    assert got["costs"]["panel"] == expect_panel
    assert (got["rows"] == ref["rows"]).all() and (got["cols"] == ref["cols"]).all()
    assert (got["offsets"] == ref["offsets"]).all()
    assert np.isfinite(got["data"]).all()
    assert rel_fro(got["data"], ref["data"]) <= tol
    return got, ref


def per_block_max_err(got, ref, row_sizes, col_sizes):
    worst = 0.0
    for b in range(len(ref["rows"])):
        n = int(row_sizes[ref["rows"][b]]) * int(col_sizes[ref["cols"][b]])
        o = int(ref["offsets"][b])
        r = ref["data"][o:o + n]
        nr = np.linalg.norm(r)
        if nr > 0:
            worst = max(worst, float(np.linalg.norm(got["data"][o:o + n] - r) / nr))
    return worst


def _mixed(seed, nb=(40, 30, 45), occ=0.25, sizes=(5, 13, 23), cin=False, alpha=1.0,
           beta=0.0, eps=0.0, ta="N", tb="N", scales=0.0, integers=False):
    rng = np.random.default_rng(seed)
    s = np.asarray(sizes, np.int32)
    m, k, n = (rng.choice(s, c).astype(np.int32) for c in nb)
    A = random_matrix(rng, m, k, occ)
    B = random_matrix(rng, k, n, occ)
    Ci = random_matrix(rng, m, n, occ * 0.6) if cin else None
    for X in (A, B):
        if integers:
            X.data[:] = rng.integers(-3, 4, X.data.size)
        elif scales:
            X.data *= np.repeat(10.0 ** -rng.uniform(0, scales, X.nblocks), X.block_lens)
    if ta == "T":
        A = transpose_matrix(A)
    if tb == "T":
        B = transpose_matrix(B)
    return Problem(A, B, Ci, alpha, beta, eps, ta, tb)


def test_panel_banded_with_filter():
    p = banded(seed=31, nb=400, decay=40.0, value_decay=8.0, eps=1e-8)
    got, ref = check(p)
    assert ref["nfiltered"] > 0
    assert got["costs"]["tensor_flops"] > 0 and got["costs"]["intermediate_bytes"] > 0


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_panel_transposes_alpha_beta_cin(ta, tb):
    # C_in has blocks that no product reaches (C = beta C_in there) and blocks shared
    # with single products (which then go through the slot reduction)
    check(_mixed(32, ta=ta, tb=tb, cin=True, alpha=-0.5, beta=2.0))


def test_panel_integer_inputs_bit_exact():
    p = _mixed(33, integers=True, cin=True, alpha=1.0, beta=-1.0)
    ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps)
    got = run_emu(p)
    assert got["costs"]["panel"]
    assert (got["data"] == ref["data"]).all()


def test_panel_block_scales_per_block_accuracy():
    """Block scales over eight decades: every C block within 1e-11 of the oracle, each
    relative to its own norm (digits are scaled per stored block and every C block's
    slots are summed at that block's own scale)."""
    p = _mixed(34, scales=8.0, occ=0.3)
    got, ref = check(p)
    assert per_block_max_err(got, ref, p.A.row_sizes, p.B.col_sizes) <= TOL


def test_panel_batched_generator_per_block_accuracy():
    """Problems of the batched workload's generator (block scales 10^-U[0,8], filter
    1e-10) run one by one on the panel kernel: per-block error within 1e-11."""
    probs = batched(nprob=4, nmin=300, nmax=900, occ_min=0.02, occ_max=0.06)
    for p in probs:
        got, ref = check(p)
        assert per_block_max_err(got, ref, p.A.row_sizes, p.B.col_sizes) <= TOL


def test_panel_repeat_bitwise_and_matches_block_kernel():
    import torch
    p = banded(seed=35, nb=300, eps=1e-8)
    got = run_emu(p)
    plan, C = got["plan"], got["C"]
    n = C.info[3]
    with panel_mode(2):
        plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
    again = C.data[:n].cpu().numpy()
    assert (again == got["data"]).all()
    old = run_emu(p, mode=0)
    assert not old["costs"]["panel"]
    assert rel_fro(got["data"], old["data"]) <= 2 * TOL


def test_panel_empty_and_filtered_everything():
    rng = np.random.default_rng(36)
    s = np.full(8, 13, np.int32)
    A = BSMatrix(s, s, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = random_matrix(rng, s, s, 0.5)
    Ci = random_matrix(rng, s, s, 0.5)
    # no product at all, C_in only: C = beta C_in
    got = run_emu(Problem(A, B, Ci, 1.0, 3.0))
    ref = oracle.multiply(A, B, Ci, 1.0, 3.0, 0.0)
    assert rel_fro(got["data"], ref["data"]) <= TOL
    # every product filtered
    p = _mixed(37, eps=1e30)
    got = run_emu(p)
    assert got["stats"]["n_stack"] == 0 and len(got["rows"]) == 0


def test_panel_not_taken_for_large_blocks():
    """n = 40 exceeds the kernel's 32-column tiles: the C-block kernel runs instead."""
    check(_mixed(38, sizes=(5, 13, 40), nb=(20, 20, 20)), expect_panel=False)


def _lib_plans(probs):
    mats, plans = [], []
    for p in probs:
        A, B = to_lib(p.A), to_lib(p.B)
        Ci = to_lib(p.C_in) if p.C_in is not None else None
        plan = bst.multiply_plan(A, B, Ci, p.eps, p.transa, p.transb)
        plan.alloc_result()
        mats.append((A, B, Ci))
        plans.append(plan)
    return mats, plans


def _plan_data(plan):
    n = plan.result.info[3]
    return plan.result.data[:n].cpu().numpy().copy()


def test_panel_batch_mixed_plans_against_oracle_and_single():
    """A batch whose plans are partly on the panel kernel (one launch over all their
    units) and partly not (blocks of 40 > 32): every plan within 1e-11 of the oracle
    per C block, bitwise equal to the same plan executed alone (each unit's digit
    products and slot sums do not depend on which other units share the launch)."""
    import torch
    probs = batched(nprob=5, nmin=300, nmax=900, occ_min=0.02, occ_max=0.06, seed=41)
    probs.append(_mixed(42, sizes=(5, 13, 40), nb=(20, 20, 20), cin=True, beta=0.5))
    probs.append(_mixed(43, ta="T", tb="T", cin=True, alpha=-0.5, beta=2.0))
    with panel_mode(2):
        mats, plans = _lib_plans(probs)
        alphas = np.array([p.alpha for p in probs])
        betas = np.array([p.beta for p in probs])
        batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
        on_panel = [bst.bst_plan_emu_costs(pl.handle)["panel"] for pl in plans]
        assert on_panel[-2] is False and sum(on_panel) == len(plans) - 1
        for pl in plans:
            pl.result.data.fill_(float("nan"))
        bst.bst_batch_execute(batch, alphas, betas, bst.BST_FP64_EMU_BF16)
        torch.cuda.synchronize()
        for pl in plans:
            assert pl.stats()["n_stack"] >= 0  # raises on a device-side timeout
        got = [_plan_data(pl) for pl in plans]
        for q, pl in enumerate(plans):
            pl.execute(alphas[q], betas[q], bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
        single = [_plan_data(pl) for pl in plans]
        bst.bst_batch_destroy(batch)
    for q, p in enumerate(probs):
        assert (got[q] == single[q]).all(), q
        ref = oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, p.transa, p.transb)
        assert rel_fro(got[q], ref["data"]) <= TOL
        if p.transa == "N" and p.transb == "N":
            g = dict(data=got[q])
            assert per_block_max_err(g, ref, p.A.row_sizes, p.B.col_sizes) <= TOL, q


def test_panel_batch_graph_replay_with_new_values():
    """The batch's panel launch captured into a CUDA graph: a replay after the operands
    changed in place reads the current data (slicing, launch and reduction are all
    graph nodes)."""
    import torch
    probs = batched(nprob=4, nmin=300, nmax=700, occ_min=0.03, occ_max=0.06, seed=44)
    with panel_mode(2):
        mats, plans = _lib_plans(probs)
        ones, zeros = np.ones(len(plans)), np.zeros(len(plans))
        batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
        assert all(bst.bst_plan_emu_costs(pl.handle)["panel"] for pl in plans)
        bst.bst_batch_execute(batch, ones, zeros, bst.BST_FP64_EMU_BF16)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=cs):
            bst.bst_batch_execute(batch, ones, zeros, bst.BST_FP64_EMU_BF16, stream=cs)
        for (A, B, _), p in zip(mats, probs):
            A.data.mul_(-2.0)  # scales every block norm alike: the filter keeps its choices
            p.A.data *= -2.0
            B.data.mul_(0.25)
            p.B.data *= 0.25
        for pl in plans:
            pl.result.data.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        got = [_plan_data(pl) for pl in plans]
        bst.bst_batch_destroy(batch)
    for q, p in enumerate(probs):
        ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps * 0.5)
        assert rel_fro(got[q], ref["data"]) <= TOL


def test_default_mode_batch_and_second_execute_per_block_accuracy():
    """The default choice (BST_TUNE_EMU_PANEL = 1) on the batched generator: a batch puts
    every plan on the panel kernel and holds 1e-11 on every C block; a plan executed on
    its own runs the C-block kernel first and the panel kernel from its second execute
    on, which then holds the same per-block bound."""
    import torch
    probs = batched(nprob=6, nmin=200, nmax=800, occ_min=0.01, occ_max=0.06, seed=45)
    with panel_mode(1):
        mats, plans = _lib_plans(probs)
        batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
        assert all(bst.bst_plan_emu_costs(pl.handle)["panel"] for pl in plans)
        ones, zeros = np.ones(len(plans)), np.zeros(len(plans))
        bst.bst_batch_execute(batch, ones, zeros, bst.BST_FP64_EMU_BF16)
        torch.cuda.synchronize()
        got = [_plan_data(pl) for pl in plans]
        bst.bst_batch_destroy(batch)
        p = probs[-1]
        A, B = to_lib(p.A), to_lib(p.B)
        plan = bst.multiply_plan(A, B, None, p.eps)
        plan.alloc_result()
        # the costs describe the next execute: here the first one
        first_on_panel = bst.bst_plan_emu_costs(plan.handle)["panel"]
        plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
        assert bst.bst_plan_emu_costs(plan.handle)["panel"]
        plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
        torch.cuda.synchronize()
        second = _plan_data(plan)
        assert bst.bst_plan_emu_costs(plan.handle)["panel"]
    assert not first_on_panel
    for q, p in enumerate(probs):
        ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
        assert per_block_max_err(dict(data=got[q]), ref, p.A.row_sizes, p.B.col_sizes) <= TOL
    assert (second == got[-1]).all()


def test_graph_capture_before_and_after_the_schedule_exists():
    """Default choice: an emulated execute captured into a CUDA graph before the panel
    schedule exists runs the C-block kernel (building the schedule would synchronise);
    once a plain execute has built it, a captured execute runs the panel kernel.  Both
    replays against the oracle."""
    import torch
    p = banded(seed=46, nb=300, eps=1e-8)
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    with panel_mode(1):
        A, B = to_lib(p.A), to_lib(p.B)
        plan = bst.multiply_plan(A, B, None, p.eps)
        C = plan.alloc_result()
        n = C.info[3]
        plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)  # first: C-block kernel state
        torch.cuda.synchronize()
        graphs = []
        for _ in range(2):
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream()
            with torch.cuda.graph(g, stream=cs):
                plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1, stream=cs)
            C.data.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            got = C.data[:n].cpu().numpy()
            assert np.isfinite(got).all()
            assert rel_fro(got, ref["data"]) <= TOL
            graphs.append(g)
            # a plain execute: builds the schedule (after the first graph)
            plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
            torch.cuda.synchronize()
        assert bst.bst_plan_emu_costs(plan.handle)["panel"]
        assert plan.stats()["n_stack"] > 0


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    """A device wait that cannot complete (an mbarrier nothing arrives at) gives up after
    its bound and is reported as BST_ERR_TIMEOUT; the next product on the same context
    still runs and matches the oracle.  No GPU fault is involved: the kernel returns."""
    import time

    import torch
    ctx = bst.context()
    t0 = time.perf_counter()
    with pytest.raises(bst.BstError) as e:
        bst.bst_debug_wait_probe(ctx, 20_000_000)  # 20 ms
    assert e.value.name == "BST_ERR_TIMEOUT"
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(bst.BstError) as e:
        bst.bst_debug_wait_probe(ctx, 10)  # below the accepted range
    assert e.value.name == "BST_ERR_INVALID_ARG"
    got, ref = check(_mixed(47), mode=2)
    assert got["stats"]["n_stack"] > 0
    torch.cuda.synchronize()
