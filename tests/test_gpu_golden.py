"""The CUDA path on the golden fixtures of tests/golden/ (integer-valued problems whose
results are exact in FP64): native FP64 reproduces every stored pattern, stack entry
and value bit for bit, with and without a K split; the emulated-FP64 and 3xTF32 paths
are held to their error bounds (1e-11, 1e-5) against the same stored values."""
import glob
import json
import os

import numpy as np
import pytest

from gpu_util import rel_fro, require_gpu
from paper_1910_13555_gb300 import bst

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MULT = sorted(glob.glob(os.path.join(GOLDEN, "multiply_*.json")))
CONT = sorted(glob.glob(os.path.join(GOLDEN, "contract_*.json")))
TOL = {bst.BST_FP64: 0.0, bst.BST_FP64_EMU_BF16: 1e-11, bst.BST_TF32X3: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def load(path):
    with open(path) as f:
        return json.load(f)


def mat(d):
    if d is None:
        return None
    return bst.Matrix.from_host(np.asarray(d["row_sizes"], np.int32),
                                np.asarray(d["col_sizes"], np.int32),
                                np.asarray(d["rows"], np.int32), np.asarray(d["cols"], np.int32),
                                np.asarray(d["data"], np.float64))


def ten(d):
    bs = [np.asarray(s, np.int32) for s in d["block_sizes"]]
    return bst.Tensor.from_host(bs, np.asarray(d["index"], np.int32).reshape(-1, len(bs)),
                                np.asarray(d["data"], np.float64))


def check(got, want, prec):
    if TOL[prec] == 0.0:
        assert np.array_equal(got, want)
    else:
        assert rel_fro(got, want) <= TOL[prec]


@pytest.mark.parametrize("split_k", [1, 3])
@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("path", MULT, ids=os.path.basename)
def test_multiply_golden(path, prec, split_k):
    import torch
    if split_k > 1 and prec != bst.BST_FP64:
        pytest.skip("the K split is a native-FP64 path")
    g = load(path)
    e = g["expected"]
    A, B, Ci = mat(g["A"]), mat(g["B"]), mat(g["C_in"])
    plan = bst.multiply(A, B, Ci, g["alpha"], g["beta"], g["eps"], g["transa"], g["transb"],
                        prec, split_k)
    torch.cuda.synchronize()
    rows, cols, offs = plan.result.index()
    assert rows.tolist() == e["rows"] and cols.tolist() == e["cols"]
    assert offs.tolist() == e["offsets"]
    st = plan.stacks()
    assert st["mnk"].ravel().tolist() == np.asarray(e["mnk"]).ravel().tolist()
    for k in ("bucket_ptr", "a_off", "b_off", "c_off"):
        assert st[k].tolist() == e[k], k
    assert plan.stats()["n_filtered"] == e["nfiltered"]
    n = plan.result.info[3]
    check(plan.result.data[:n].cpu().numpy(), np.asarray(e["data"], np.float64), prec)


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("path", CONT, ids=os.path.basename)
def test_contract_golden(path, prec):
    import torch
    g = load(path)
    e = g["expected"]
    plan = bst.contract(ten(g["T1"]), ten(g["T2"]), g["c1"], g["c2"], g["f1"], g["f2"],
                        g["result_order"], ten(g["R_in"]), g["alpha"], g["beta"], g["eps"], prec)
    torch.cuda.synchronize()
    idx, off = plan.result.index()
    assert idx.ravel().tolist() == np.asarray(e["index"]).ravel().tolist()
    assert off.tolist() == e["offsets"]
    assert plan.stats()["n_stack"] == e["npairs"]
    n = plan.result.info[2]
    check(plan.result.data[:n].cpu().numpy(), np.asarray(e["data"], np.float64), prec)
