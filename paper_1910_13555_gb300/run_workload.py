"""Run one of the synthetic workloads through the library a few times (a driver for
profilers and quick timings).

    python -m paper_1910_13555_gb300.run_workload <name> [--reps N] [--precision P] [--nb N] [--np P]
                                                        [--adjoint] [--emu-kernel K]

name: banded | tall_skinny | rect_case2 | batched | rank3 | rank4 | sign
precision: fp64 | emu | tf32x3
emu-kernel (emulated FP64): auto (default choice) | panel (the tcgen05 panel kernel when the
blocks fit) | block (the C-block kernel)

Each run builds the plan once and executes it `reps` times (a batch for `batched`,
one Newton-Schulz step for `sign`, the adjoint dT, dU with --adjoint for `rank3` and
`rank4`), then prints the flop count and the median CUDA-event time of the executes.
"""
from __future__ import annotations

import argparse
import statistics
import sys

PRECISIONS = {"fp64": "BST_FP64", "emu": "BST_FP64_EMU_BF16", "tf32x3": "BST_TF32X3"}


def main(argv=None) -> int:
    import numpy as np
    import torch

    from . import bst, sign, workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=["banded", "tall_skinny", "rect_case2", "batched", "rank3",
                                     "rank4", "sign"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS))
    ap.add_argument("--nb", type=int, default=None, help="banded / sign: blocks per side")
    ap.add_argument("--np", type=int, default=None,
                    help="rank3 / rank4: P blocks (fewer products per C block, same C pattern)")
    ap.add_argument("--adjoint", action="store_true",
                    help="rank3 / rank4: time the adjoint (dT, dU from dR = R) instead")
    ap.add_argument("--emu-kernel", default="auto", choices=["auto", "panel", "block"])
    a = ap.parse_args(argv)
    prec = getattr(bst, PRECISIONS[a.precision])
    bst.bst_tune_set(bst.context(), bst.BST_TUNE_EMU_PANEL,
                     {"auto": 1, "panel": 2, "block": 0}[a.emu_kernel])

    def mk(m):
        return bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data)

    keep = []
    if a.name in ("banded", "tall_skinny", "rect_case2"):
        p = {"banded": lambda: workloads.banded(nb=a.nb or 4000),
             "tall_skinny": workloads.tall_skinny, "rect_case2": workloads.rect_case2}[a.name]()
        A, B = mk(p.A), mk(p.B)
        plan = bst.multiply_plan(A, B, None, p.eps, p.transa, p.transb)
        plan.alloc_result()
        keep = [A, B, plan]
        flops = plan.stats()["flops"]
        run = lambda: plan.execute(1.0, 0.0, prec, 1)  # noqa: E731
    elif a.name in ("rank3", "rank4"):
        kw = {} if a.np is None else {"nP": a.np}
        w = workloads.rank3(**kw) if a.name == "rank3" else workloads.rank4(**kw)
        t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data)
        t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data)
        plan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, precision=prec)
        keep = [t1, t2, plan]
        flops = plan.stats()["flops"]
        run = lambda: plan.execute(1.0, 0.0, prec, 1)  # noqa: E731
        if a.adjoint:
            torch.cuda.synchronize()
            ne = plan.result.info[2]
            dR = plan.result.data[:ne].clone()
            dT, dU = torch.empty_like(t1.data), torch.empty_like(t2.data)
            keep += [dR, dT, dU]
            flops = 2.0 * flops
            run = lambda: bst.bst_plan_adjoint(plan.handle, dR, dT, dU, None, 1.0, 0.0)  # noqa: E731
    elif a.name == "batched":
        probs = workloads.batched()
        plans = []
        for q in probs:
            A, B = mk(q.A), mk(q.B)
            pl = bst.multiply_plan(A, B, None, q.eps)
            pl.alloc_result()
            keep += [A, B]
            plans.append(pl)
        batch = bst.bst_batch_create(bst.context(), [pl.handle for pl in plans])
        keep += plans
        ones, zeros = np.ones(len(plans)), np.zeros(len(plans))
        flops = sum(pl.stats()["flops"] for pl in plans)
        run = lambda: bst.bst_batch_execute(batch, ones, zeros, prec)  # noqa: E731
    else:
        X = mk(workloads.sign_matrix(nb=a.nb or 2000))
        keep = [X]
        st = {}

        def run():
            _, s = sign.sign_step(X, precision=prec)
            st.update(s)
        run()
        flops = st["flops"]
    run()
    torch.cuda.synchronize()
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    times = []
    for _ in range(a.reps):
        ev[0].record()
        run()
        ev[1].record()
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    ms = statistics.median(times) if times else float("nan")
    print(f"{a.name} {a.precision}: {flops:.4e} flop, {ms:.3f} ms, "
          f"{flops / (ms * 1e-3) / 1e9:.1f} GFLOP/s", flush=True)
    del keep
    return 0


if __name__ == "__main__":
    sys.exit(main())
