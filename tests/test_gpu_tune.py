"""The autotuner's per-(m, n) tile mapping of the emulated-FP64 kernel: every mapping
gives results within 1e-11 of the oracle, and the tuner leaves a valid choice set."""
import numpy as np
import pytest

import oracle
from gpu_util import rel_fro, require_gpu, to_lib
from paper_1910_13555_gb300 import bst, tune
from paper_1910_13555_gb300.workloads import banded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture()
def ctx():
    c = bst.context()
    yield c
    for m in (5, 7, 13, 23, 31):
        for n in (5, 7, 13, 23, 31):
            bst.bst_tune_set(c, bst.BST_TUNE_EMU_SWAP, -1, m, n)


def _problem():
    p = banded(seed=21, nb=240, decay=40.0, value_decay=8.0, eps=1e-8)
    return p


@pytest.mark.parametrize("force", [0, 1])
def test_every_mapping_is_exact_enough(ctx, force):
    import torch
    p = _problem()
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps)
    C = plan.alloc_result()
    for (m, n) in tune.plan_classes(plan):
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_SWAP, force, m, n)
    plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
    torch.cuda.synchronize()
    n_el = C.info[3]
    assert rel_fro(C.data[:n_el].cpu().numpy(), ref["data"]) <= 1e-11


def test_tuner_sets_choices_and_round_trips(ctx, tmp_path):
    import torch
    p = _problem()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps)
    C = plan.alloc_result()
    table = tune.tune_emulated(plan, reps=2)
    assert set(table) == set(tune.plan_classes(plan))
    for (m, n), v in table.items():
        assert bst.bst_tune_get(ctx, bst.BST_TUNE_EMU_SWAP, m, n) == v["swap"]
        assert v["ms"][v["swap"]] == min(v["ms"].values())
    path = str(tmp_path / "tune.json")
    tune.save_table(table, path, "gpu-x")
    for (m, n) in table:
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_SWAP, -1, m, n)
    again = tune.load_table(path, "gpu-x")
    assert {k: v["swap"] for k, v in again.items()} == {k: v["swap"] for k, v in table.items()}
    # results after tuning still match the oracle
    plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1)
    torch.cuda.synchronize()
    ref = oracle.multiply(p.A, p.B, None, 1.0, 0.0, p.eps)
    assert rel_fro(C.data[:C.info[3]].cpu().numpy(), ref["data"]) <= 1e-11


def test_batch_refuses_after_retune(ctx):
    p = _problem()
    A, B = to_lib(p.A), to_lib(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps)
    plan.alloc_result()
    batch = bst.bst_batch_create(ctx, [plan.handle])
    bst.bst_batch_execute(batch, [1.0], [0.0], bst.BST_FP64_EMU_BF16)
    m, n = tune.plan_classes(plan)[0]
    bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_SWAP, 1, m, n)
    with pytest.raises(bst.BstError) as e:
        bst.bst_batch_execute(batch, [1.0], [0.0], bst.BST_FP64_EMU_BF16)
    assert e.value.name == "BST_ERR_STATE"
    bst.bst_batch_execute(batch, [1.0], [0.0], bst.BST_FP64)  # native FP64 is unaffected
    bst.bst_batch_destroy(batch)
