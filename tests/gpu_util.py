"""Helpers of the GPU tests: move workload inputs into the library and results back."""
from __future__ import annotations

import numpy as np

from paper_1910_13555_gb300 import bst


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is visible")
    bst.load()


def to_lib(m):
    return bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)


def rel_fro(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def run_multiply(p, precision=bst.BST_FP64, split_k=1, stacks=True):
    import torch
    A, B = to_lib(p.A), to_lib(p.B)
    Ci = to_lib(p.C_in) if p.C_in is not None else None
    plan = bst.multiply(A, B, Ci, p.alpha, p.beta, p.eps, p.transa, p.transb, precision, split_k)
    torch.cuda.synchronize()
    rows, cols, offs = plan.result.index()
    nelem = plan.result.info[3]
    out = dict(rows=rows, cols=cols, offsets=offs,
               data=plan.result.data[:nelem].cpu().numpy(), stats=plan.stats(), plan=plan,
               mats=(A, B, Ci))
    if stacks:
        out.update(plan.stacks())
    return out
