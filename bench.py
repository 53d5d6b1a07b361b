#!/usr/bin/env python3
"""Benchmark of the block-sparse multiply on one GB300 per rank.

Workload: the banded product (4000 x 4000 blocks of sizes {5:40%, 13:40%, 23:20%},
~1 % occupancy with block (i,j) kept w.p. c*exp(-|i-j|/200), entries
N(0,1)*exp(-|i-j|/50), norm filter eps = 1e-8, C = A*B, beta = 0), synthetic and
seeded.  One step = one pass of the whole path on the GPU with inputs resident in
HBM: block norms, symbolic phase (pair matching + filter, C pattern, stacks), C_out
allocation, numeric phase.  `value` is the whole-job GFLOP/s (sum over ranks of the
algorithmic flops 2*m*n*k of every kept product / max over ranks of the timed span).

With torchrun (N > 1) every rank runs its own independent product (seed 1002 +
1000*rank): the work is partitioned across ranks with no data-path collective
(weak scaling).  `--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block-sparse multiply GFLOP/s & roofline fraction: FP64 vs emulated-FP64 @1e-11"
UNIT = "GFLOP/s"
WORKLOAD = ("banded 4000x4000 blocks, sizes {5:.4,13:.4,23:.2}, ~1% occupancy "
            "(keep w.p. c*exp(-|i-j|/200)), entries N(0,1)*exp(-|i-j|/50), eps=1e-8, C=A*B")
# FP64 FMA peak of one GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM
# x 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _measured_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("bf16_tflops") or 0.0) or None
    except (OSError, ValueError, TypeError):
        return None


BF16_PEAK_TFLOPS = _measured_bf16()
CPU_SAMPLE_ROWS = (1000, 3000)     # cpu_baseline: block rows of A in the sample
REF_SAMPLE_ROWS = (1800, 2200)     # --impl reference: block rows per step
# timed-step precision -> (library constant name, numeric kernel launched by execute)
PRECISIONS = {"fp64": ("BST_FP64", "k_num_fp64_staged1"),
              "emu": ("BST_FP64_EMU_BF16", "k_num_emu_bf16_persist1"),
              "tf32x3": ("BST_TF32X3", "k_num_tf32x3")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the precision-variant legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nb", type=int, default=4000,
                    help="block rows/columns of the banded workload (smaller for profiler captures)")
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS),
                    help="precision of the timed step (the headline is native fp64)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------


def load_traffic(kernel_tag):
    """DRAM bytes per launch of the kernel from the committed ncu summary, if present."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("traffic_bytes_per_launch:"):
            v = line.split(":", 1)[1].strip()
            return None if v in ("", "null") else float(v)
    return None


def cpu_baseline(p, rows, steps=1):
    """Time the CPU oracle (single thread, as it stands) on a sample of block rows."""
    import numpy as np

    import oracle
    from paper_1910_13555_gb300.workloads import BSMatrix

    oracle.build()
    r0, r1 = rows
    sel = (p.A.rows >= r0) & (p.A.rows < r1)
    offs, lens = p.A.offsets, p.A.block_lens
    idx = np.concatenate([np.arange(offs[b], offs[b] + lens[b]) for b in np.nonzero(sel)[0]])
    A2 = BSMatrix(p.A.row_sizes, p.A.col_sizes, p.A.rows[sel], p.A.cols[sel], p.A.data[idx])
    times, flops = [], 0.0
    for _ in range(steps):
        t = time.perf_counter()
        res = oracle.multiply(A2, p.B, None, 1.0, 0.0, p.eps)
        times.append(time.perf_counter() - t)
        flops = res["flops"]
    return flops, times


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from paper_1910_13555_gb300.workloads import banded
    p = banded()
    if args.warmup > 0:
        cpu_baseline(p, REF_SAMPLE_ROWS, steps=args.warmup)
    flops, times = cpu_baseline(p, REF_SAMPLE_ROWS, steps=args.steps)
    total = sum(times)
    value = flops * args.steps / total / 1e9
    sample = f"block rows {REF_SAMPLE_ROWS[0]}..{REF_SAMPLE_ROWS[1]} of A (all of B), {flops:.3e} flop per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample, "parallelism": "cpu oracle, 1 thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# measured BF16 mma.sync throughput of one GB300 (a throughput probe with 8 independent
# chains per thread); the emulated kernel is built on mma.sync m16n8k16
MMA_SYNC_BF16_TFLOPS = 604.0


def emu_tensor_ops(plan, ctx):
    """BF16 tensor flops the emulated kernel executes for a plan: per product 21 slice
    products on 16 x 8 tiles covering the C block (rows over the block's rows, or over
    its columns for a swapped class) and the inner size padded to 16."""
    from paper_1910_13555_gb300 import bst
    st = bst.bst_plan_get_stacks(plan.handle)
    cnt = (st["bucket_ptr"][1:] - st["bucket_ptr"][:-1]).astype(float)
    total = 0.0
    for (m, n, k), c in zip(st["mnk"].tolist(), cnt):
        sw = bst.bst_tune_get(ctx, bst.BST_TUNE_EMU_SWAP, m, n)
        plain = -(-m // 16) * -(-n // 8)
        swapped = -(-n // 16) * -(-m // 8)
        if sw < 0:
            sw = 1 if swapped < plain else 0
        tiles = swapped if sw else plain
        total += c * 21 * 2 * tiles * 16 * 8 * 16 * -(-k // 16)
    return total


def keep_plan_index(A, B, p, device):
    """C block index of the workload's product (rows, cols, offsets) from one plan."""
    from paper_1910_13555_gb300 import bst
    plan = bst.multiply_plan(A, B, None, p.eps, device=device)
    r, c, o = bst.bst_matrix_get_index(bst.bst_plan_result(plan.handle))
    return r, c, o


class SampledError:
    """Relative Frobenius error of a result on 64 seeded C blocks against the CPU oracle
    (the oracle computes exactly those blocks from the definition)."""

    def __init__(self, p, index, nsample=64, seed=0):
        import numpy as np

        import oracle
        rows, cols, offs = index
        rng = np.random.default_rng(seed)
        self.sel = np.sort(rng.choice(len(rows), min(nsample, len(rows)), replace=False))
        self.bi, self.bj, self.offs = rows[self.sel], cols[self.sel], offs[self.sel]
        self.m = p.A.row_sizes[self.bi].astype(np.int64)
        self.n = p.B.col_sizes[self.bj].astype(np.int64)
        self.ref, _ = oracle.multiply_sample(p.A, p.B, None, 1.0, 0.0, p.eps, self.bi, self.bj,
                                             row_sizes=p.A.row_sizes, col_sizes=p.B.col_sizes)

    def error(self, plan):
        import numpy as np
        import torch
        d = plan.result.data
        idx = np.concatenate([np.arange(o, o + m * n) for o, m, n in zip(self.offs, self.m, self.n)])
        got = d[torch.as_tensor(idx, device=d.device)].cpu().numpy()
        return float(np.linalg.norm(got - self.ref) / np.linalg.norm(self.ref))

    def describe(self):
        return f"{len(self.sel)} seeded C blocks ({int((self.m * self.n).sum())} elements)"


def run_ours(args):
    import numpy as np
    import torch

    from paper_1910_13555_gb300 import bst
    from paper_1910_13555_gb300.workloads import banded

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    bst.load()
    p = banded(seed=1002 + 1000 * rank, nb=args.nb)
    workload = WORKLOAD if args.nb == 4000 else WORKLOAD.replace("4000x4000", f"{args.nb}x{args.nb}")
    prec_name, kernel = PRECISIONS[args.precision]
    main_prec = getattr(bst, prec_name)
    mk = lambda m: bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data,
                                        device=local_rank)
    A, B = mk(p.A), mk(p.B)
    stream = torch.cuda.current_stream()

    def step(precision=main_prec, events=None):
        plan = bst.multiply_plan(A, B, None, p.eps, device=local_rank)
        plan.alloc_result(local_rank)
        if events is not None:
            events[0].record(stream)
        plan.execute(1.0, 0.0, precision, 1)
        if events is not None:
            events[1].record(stream)
        return plan

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        keep = step()
    barrier()
    flops = keep.stats()["flops"]
    stats = keep.stats()
    c_bytes = 8 * int(keep.result.info[3])
    del keep
    ab_bytes = p.A.data.nbytes + p.B.data.nbytes
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = bst.bst_kernel_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    plans = []
    t0.record(stream)
    for k in range(args.steps):
        plans.append(step(events=evs[k]))
        if len(plans) > 2:
            plans.pop(0)
    t1.record(stream)
    barrier()
    launches = bst.bst_kernel_launches() - l0
    clk = clocks.stop()
    plans.clear()
    ms = t0.elapsed_time(t1)
    num_ms = [a.elapsed_time(b) for a, b in evs]
    ms_max = ms
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(t.item())
        f = torch.tensor([flops], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(f)
        total_flops = float(f.item())
    else:
        total_flops = flops
    value = total_flops * args.steps / (ms_max * 1e-3) / 1e9
    num_avg = statistics.mean(num_ms)
    achieved = flops / (num_avg * 1e-3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "emu": "bf16", "tf32x3": "tf32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload,
                   "precision": {"fp64": "native fp64", "emu": "fp64 emulated on bf16 slices",
                                 "tf32x3": "3xtf32"}[args.precision],
                   "global_batch": world,
                   "parallelism": f"{world} independent products, one per GPU",
                   "l2": f"inputs larger than L2 (A+B {ab_bytes / 1e9:.2f} GB read per step, "
                         f"C {c_bytes / 1e9:.2f} GB written)",
                   "flop_per_step_per_gpu": flops, "c_blocks": stats["n_c_blocks"],
                   "stack_entries": stats["n_stack"], "filtered": stats["n_filtered"]},
        "numeric_only": {"value": flops / (num_avg * 1e-3) / 1e9, "unit": UNIT,
                         "ms": num_avg},
        "roofline": ({"bound": "alu", "kernel": kernel, "achieved": achieved,
                      "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                      "frac": achieved / FP64_PEAK_TFLOPS,
                      "peak_note": "FP64 FMA pipe: 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz",
                      "traffic": load_traffic(f"{kernel}_banded") if args.nb == 4000 else None}
                     if args.precision == "fp64" else None),
        "gpu_launches": launches,
        "clocks": clk,
    }

    if not args.no_e2e:
        line["e2e"] = e2e_leg(p, local_rank, min(args.steps, 3), stream, barrier, world, dev)

    if not args.no_extras:
        from paper_1910_13555_gb300 import tune
        extras = {}
        sample = SampledError(p, keep_plan_index(A, B, p, local_rank)) if rank == 0 else None
        if sample is not None:
            fp = step(bst.BST_FP64)
            torch.cuda.synchronize()
            line["numeric_only"]["rel_err_vs_oracle_sample"] = sample.error(fp)
            del fp
        for name, prec in (("emu_bf16", bst.BST_FP64_EMU_BF16), ("tf32x3", bst.BST_TF32X3)):
            try:
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                pl = step(prec)
                torch.cuda.synchronize()
                if prec == bst.BST_FP64_EMU_BF16:
                    # the project's autotuner picks the tile mapping per (m, n) class
                    table = tune.tune_emulated(pl, device=local_rank, reps=2)
                    extras["emu_tuned_swap"] = {f"{m}x{n}": v["swap"] for (m, n), v in table.items()}
                # first execute of a fresh plan (builds the plan's slicing index), then
                # repeated executes of that plan (slicing of the current data + products)
                first = []
                for _ in range(2):
                    pl2 = step(prec, ev)
                    torch.cuda.synchronize()
                    first.append(ev[0].elapsed_time(ev[1]))
                times = []
                for _ in range(5):
                    ev[0].record(stream)
                    pl2.execute(1.0, 0.0, prec, 1)
                    ev[1].record(stream)
                    torch.cuda.synchronize()
                    times.append(ev[0].elapsed_time(ev[1]))
                t = statistics.median(times)
                extras[name] = {"numeric_gflops": flops / (t * 1e-3) / 1e9, "ms": t,
                                "speedup_vs_fp64_numeric": num_avg / t,
                                "first_execute_ms": min(first),
                                "note": "repeat executes of one plan; first_execute_ms adds "
                                        "the per-plan slicing index"}
                if prec == bst.BST_FP64_EMU_BF16:
                    ops = emu_tensor_ops(pl2, bst.context(local_rank))
                    achieved_t = ops / (t * 1e-3) / 1e12
                    extras[name]["tensor_roofline"] = {
                        "bound": "tensor", "executed_bf16_tflop_per_execute": ops / 1e12,
                        "achieved": achieved_t, "unit": "TFLOP/s",
                        "peak_mma_sync_bf16": MMA_SYNC_BF16_TFLOPS,
                        "frac": achieved_t / MMA_SYNC_BF16_TFLOPS,
                        "peak_measured_bf16": BF16_PEAK_TFLOPS,
                        "frac_of_measured": achieved_t / BF16_PEAK_TFLOPS if BF16_PEAK_TFLOPS else None,
                        "note": "whole execute (slicing + products) against the BF16 mma.sync "
                                "rate and the measured cuBLAS BF16 rate"}
                if sample is not None:
                    extras[name]["rel_err_vs_oracle_sample"] = sample.error(pl2)
                del pl, pl2
            except bst.BstError as e:
                extras[name] = {"unavailable": e.name}
        if sample is not None:
            extras["error_sample"] = sample.describe()
        line["precision_variants"] = extras

    if rank == 0 and world == 1 and not args.no_cpu:
        rows = CPU_SAMPLE_ROWS if args.nb == 4000 else (args.nb // 4, 3 * args.nb // 4)
        fl, times = cpu_baseline(p, rows, steps=1)
        line["cpu_baseline"] = {
            "value": fl / times[0] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"block rows {rows[0]}..{rows[1]} of A times all of B "
                      f"({fl:.3e} flop, {times[0]:.1f} s, single thread)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def e2e_leg(p, local_rank, steps, stream, barrier, world, dev):
    """The same metric through the public API from host buffers: each step creates
    the matrices from host index arrays and pinned host data (H2D inside), plans,
    executes and reads C_out back into pinned host memory (D2H inside)."""
    import numpy as np
    import torch

    from paper_1910_13555_gb300 import bst

    ha = torch.from_numpy(p.A.data).pin_memory()
    hb = torch.from_numpy(p.B.data).pin_memory()
    ctx = bst.context(local_rank)
    hc = None
    flops = 0.0

    def one():
        nonlocal hc, flops
        da = ha.to(dev, non_blocking=True)
        db = hb.to(dev, non_blocking=True)
        A = bst.Matrix(bst.bst_matrix_create(ctx, p.A.row_sizes, p.A.col_sizes, p.A.rows,
                                             p.A.cols, da), da)
        B = bst.Matrix(bst.bst_matrix_create(ctx, p.B.row_sizes, p.B.col_sizes, p.B.rows,
                                             p.B.cols, db), db)
        plan = bst.multiply(A, B, None, 1.0, 0.0, p.eps, device=local_rank)
        n = plan.result.info[3]
        if hc is None or hc.numel() < n:
            hc = torch.empty(n, dtype=torch.float64).pin_memory()
        hc[:n].copy_(plan.result.data[:n], non_blocking=True)
        torch.cuda.synchronize()
        flops = plan.stats()["flops"]
        return n

    n = one()
    barrier()
    t = time.perf_counter()
    for _ in range(steps):
        n = one()
    barrier()
    dt = (time.perf_counter() - t) / steps
    if world > 1:
        tt = torch.tensor([dt], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        dt = float(tt.item())
        f = torch.tensor([flops], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(f)
        flops = float(f.item())
    h2d = (p.A.data.nbytes + p.B.data.nbytes + 8 * (p.A.nblocks + p.B.nblocks) +
           4 * (len(p.A.row_sizes) + len(p.A.col_sizes) + len(p.B.row_sizes) + len(p.B.col_sizes)))
    return {"value": flops / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(8 * n), "ms_per_step": dt * 1e3}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
