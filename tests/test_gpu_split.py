"""Inner-dimension split of the staged native-FP64 kernel (tiles whose m n outputs leave
lanes idle spread k over s lane groups and add the partial sums in a fixed order):
every split bound gives results within 1e-12 of the oracle, the split is really taken,
results are deterministic, and the autotuner leaves valid choices."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, run_multiply, to_lib
from paper_1910_13555_gb300 import bst, tune
from paper_1910_13555_gb300.workloads import (Problem, bernoulli_pattern, make_matrix,
                                              tall_skinny)

pytestmark = pytest.mark.gpu

SIZES = (5, 7, 13, 23, 30, 40, 50)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture()
def ctx():
    c = bst.context()
    yield c
    for m in SIZES:
        for n in SIZES:
            bst.bst_tune_set(c, bst.BST_TUNE_F64_SPLIT, -1, m, n)


def _bound_all(ctx, v):
    for m in SIZES:
        for n in SIZES:
            bst.bst_tune_set(ctx, bst.BST_TUNE_F64_SPLIT, v, m, n)


def _tall_skinny():
    # A^T B, inner blocks 20..50, C blocks 5 x 5 .. 13 x 13: the split's home ground
    return tall_skinny(seed=41, nk=3000, nmn=40, window=12, p=0.3)


def _with_tiles_and_cin():
    # mostly 5 x 13 C blocks (split) beside 40 x 40 ones (row tiles of 13 rows, inner
    # panels of 50), C_in with its own pattern, alpha and beta not 1
    rng = np.random.default_rng(42)
    rsz = rng.choice(np.array([5, 5, 5, 5, 5, 5, 7, 40], np.int32), 60).astype(np.int32)
    ksz = rng.choice(np.array([30, 50], np.int32), 60).astype(np.int32)
    csz = rng.choice(np.array([13, 13, 13, 13, 40], np.int32), 60).astype(np.int32)
    A = make_matrix(rng, rsz, ksz, *bernoulli_pattern(rng, 60, 60, 0.3))
    B = make_matrix(rng, ksz, csz, *bernoulli_pattern(rng, 60, 60, 0.3))
    Ci = make_matrix(rng, rsz, csz, *bernoulli_pattern(rng, 60, 60, 0.05))
    return Problem(A, B, Ci, alpha=-0.75, beta=1.25, name="tiles+cin")


def _ref(p):
    return oracle.multiply(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, p.transa, p.transb)


@pytest.mark.parametrize("make", [_tall_skinny, _with_tiles_and_cin])
@pytest.mark.parametrize("bound", [1, 2, 16, -1])
def test_every_split_bound_matches_oracle(ctx, make, bound):
    p = make()
    _bound_all(ctx, bound)
    out = run_multiply(p, stacks=False)
    ref = _ref(p)
    assert (out["rows"] == ref["rows"]).all() and (out["cols"] == ref["cols"]).all()
    assert rel_fro(out["data"], ref["data"]) <= 1e-12
    hist = out["plan"].split_histogram()
    assert hist[0] == 0 and hist.sum() > 0
    if bound == 1:
        assert hist[2:].sum() == 0
    else:
        eff = 16 if bound == -1 else bound
        assert hist[eff + 1:].sum() == 0
        if eff == 16:
            assert hist[2:].sum() > 0  # some tile took a split


def test_split_is_deterministic_and_retunes_between_executes(ctx):
    import torch
    p = _tall_skinny()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    n = C.info[3]
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    first = C.data[:n].clone()
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    torch.cuda.synchronize()
    assert torch.equal(first, C.data[:n])
    h_auto = plan.split_histogram()
    assert h_auto[2:].sum() > 0
    _bound_all(ctx, 1)  # the next execute splits the tiles again, now not at all
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    torch.cuda.synchronize()
    h_off = plan.split_histogram()
    assert h_off[2:].sum() == 0 and h_off[1] == h_auto.sum()
    ref = _ref(p)
    assert rel_fro(C.data[:n].cpu().numpy(), ref["data"]) <= 1e-12


def test_batch_resplits_before_running(ctx):
    import torch
    p = _tall_skinny()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    batch = bst.bst_batch_create(ctx, [plan.handle])
    ref = _ref(p)
    for bound, split in ((1, False), (-1, True)):
        _bound_all(ctx, bound)
        C.data.zero_()
        bst.bst_batch_execute(batch, [1.0], [0.0], bst.BST_FP64)
        torch.cuda.synchronize()
        h = plan.split_histogram()
        assert (h[2:].sum() > 0) == split
        assert rel_fro(C.data[:C.info[3]].cpu().numpy(), ref["data"]) <= 1e-12
    bst.bst_batch_destroy(batch)


def test_tuner_sets_split_choices(ctx):
    import torch
    p = _tall_skinny()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
    C = plan.alloc_result()
    table = tune.tune_fp64_split(plan, reps=2)
    assert set(table) == set(tune.plan_classes(plan))
    for (m, n), v in table.items():
        assert v["split"] in tune.SPLIT_CHOICES
        assert bst.bst_tune_get(ctx, bst.BST_TUNE_F64_SPLIT, m, n) == v["split"]
        assert v["ms"][v["split"]] == min(v["ms"].values())
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    torch.cuda.synchronize()
    ref = _ref(p)
    assert rel_fro(C.data[:C.info[3]].cpu().numpy(), ref["data"]) <= 1e-12


def test_split_bound_rejects_bad_values(ctx):
    for v in (0, 17, -2):
        with pytest.raises(bst.BstError) as e:
            bst.bst_tune_set(ctx, bst.BST_TUNE_F64_SPLIT, v, 5, 13)
        assert e.value.name == "BST_ERR_INVALID_ARG"
    assert bst.bst_tune_get(ctx, bst.BST_TUNE_F64_SPLIT, 5, 13) == -1


def test_split_never_outgrows_a_small_slot(ctx):
    # only 5 x 5 x 5 products, ~15 per C block: a slot holds 50 doubles, fewer than the
    # 125 partial sums a 5-way split would add through it
    rng = np.random.default_rng(44)
    sz = np.full(60, 5, np.int32)
    A = make_matrix(rng, sz, sz, *bernoulli_pattern(rng, 60, 60, 0.5))
    B = make_matrix(rng, sz, sz, *bernoulli_pattern(rng, 60, 60, 0.5))
    p = Problem(A, B)
    out = run_multiply(p, stacks=False)
    ref = _ref(p)
    assert rel_fro(out["data"], ref["data"]) <= 1e-12
    hist = out["plan"].split_histogram()
    assert hist[3:].sum() == 0  # s m n <= 50
