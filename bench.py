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


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("hbm_gbs") or 0.0) or None
    except (OSError, ValueError, TypeError):
        return None


MEASURED_HBM_GBS = _measured_hbm()
CPU_SAMPLE_ROWS = (1000, 3000)     # cpu_baseline: block rows of A in the sample
D2H_SPLIT = 4                      # e2e: parts of C's read-back, one copy stream each
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
    ap.add_argument("--no-cpu-parallel", action="store_true",
                    help="skip the multi-process leg of the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (tiny, tall-skinny, batched, rank-3)")
    ap.add_argument("--nb", type=int, default=4000,
                    help="block rows/columns of the banded workload (smaller for profiler captures)")
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS),
                    help="precision of the timed step (the headline is native fp64)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def rank_seed(rank):
    """Each rank multiplies its own banded product (the path partitions into independent
    problems: no data-path collective, weak scaling)."""
    return 1002 + 1000 * rank


def reduce_over_ranks(ms, flops, world, device):
    """Whole-job timing: the slowest rank's time and the work of all ranks (the only
    collectives of the benchmark, after the timed region)."""
    if world <= 1:
        return ms, flops
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    f = torch.tensor([flops], device=device, dtype=torch.float64)
    dist.all_reduce(f)
    return float(t.item()), float(f.item())


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


def _oracle_rows_worker(seed, nb, r0, r1, barrier, queue):
    """One process of the parallel CPU baseline: the oracle on block rows [r0, r1) of A
    (its own copy of the workload, built before the common start)."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle
    from paper_1910_13555_gb300.workloads import BSMatrix, banded
    p = banded(seed=seed, nb=nb)
    sel = (p.A.rows >= r0) & (p.A.rows < r1)
    offs, lens = p.A.offsets, p.A.block_lens
    idx = np.concatenate([np.arange(offs[b], offs[b] + lens[b]) for b in np.nonzero(sel)[0]])
    A2 = BSMatrix(p.A.row_sizes, p.A.col_sizes, p.A.rows[sel], p.A.cols[sel], p.A.data[idx])
    barrier.wait(timeout=600)
    t0 = time.time()
    res = oracle.multiply(A2, p.B, None, 1.0, 0.0, p.eps)
    queue.put((res["flops"], t0, time.time()))


def cpu_baseline_parallel(seed, nb, rows, workers):
    """The oracle, as it stands, in `workers` processes over disjoint ranges of block rows
    of A (the parallel leg of the CPU baseline); wall time from the common start to the
    last finish."""
    import multiprocessing as mp

    import numpy as np

    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(workers), ctx.Queue()
    bounds = np.linspace(rows[0], rows[1], workers + 1).astype(int)
    procs = [ctx.Process(target=_oracle_rows_worker,
                         args=(seed, nb, int(bounds[i]), int(bounds[i + 1]), barrier, queue))
             for i in range(workers)]
    for pr in procs:
        pr.start()
    out, deadline = [], time.time() + 900
    try:
        while len(out) < workers:
            try:
                out.append(queue.get(timeout=1.0))
            except Exception:
                bad = [pr.exitcode for pr in procs if pr.exitcode not in (None, 0)]
                if bad or time.time() > deadline:
                    raise RuntimeError(f"parallel oracle baseline failed (exit codes {bad})")
    finally:
        for pr in procs:
            pr.join(timeout=5)
            if pr.is_alive():
                pr.terminate()
    flops = sum(o[0] for o in out)
    return flops, max(o[2] for o in out) - min(o[1] for o in out)


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


def emu_roofline(plans, ms, ctx):
    """Roofline of the emulated-FP64 execute of `plans` (run together in `ms`): the time
    the slice products would take at the measured BF16 peak against the time its bytes
    would take at the measured HBM bandwidth; fraction = the larger / measured time.
    Executed tensor flops and bytes come from the library (bst_plan_emu_costs)."""
    from paper_1910_13555_gb300 import bst
    ops = byt = inter = 0.0
    for pl in plans:
        c = bst.bst_plan_emu_costs(pl.handle)
        ops += c["tensor_flops"]
        byt += c["bytes"]
        inter += c["intermediate_bytes"]
    hbm = MEASURED_HBM_GBS
    t_tensor = ops / (BF16_PEAK_TFLOPS * 1e12) if BF16_PEAK_TFLOPS else 0.0
    t_hbm = byt / (hbm * 1e9) if hbm else 0.0
    t_roof = max(t_tensor, t_hbm)
    t_roof2 = max(t_tensor, (byt + inter) / (hbm * 1e9) if hbm else 0.0)
    return {"bound": "tensor" if t_tensor >= t_hbm else "hbm",
            "executed_bf16_tflop": ops / 1e12, "bytes": byt, "intermediate_bytes": inter,
            "t_roof_ms": t_roof * 1e3, "frac": t_roof / (ms * 1e-3) if ms > 0 else None,
            "frac_with_intermediates": t_roof2 / (ms * 1e-3) if ms > 0 else None,
            "peaks": f"bf16 {BF16_PEAK_TFLOPS} TFLOP/s, hbm {hbm} GB/s (measured)",
            "note": "bytes: operands read by the slicing passes, digit planes written and "
                    "read once, C written, schedule read; intermediate_bytes: partial "
                    "products written and read back (the panel path's int64 slots)"}


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
    p = banded(seed=rank_seed(rank), nb=args.nb)
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

    keep = None
    for _ in range(max(args.warmup, 0)):
        keep = step()
    if keep is None:  # no warm-up asked for: the plan alone (symbolic phase) for the counts
        keep = bst.multiply_plan(A, B, None, p.eps, device=local_rank)
        keep.alloc_result(local_rank)
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
    ms_max, total_flops = reduce_over_ranks(ms, flops, world, dev)
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
                         "ms": num_avg, "ms_median": statistics.median(num_ms),
                         "launches_timed": len(num_ms)},
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
        line["e2e"] = e2e_leg(p, local_rank, max(args.steps, 20), stream, barrier, world, dev)

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
                pl2.execute(1.0, 0.0, prec, 1)  # second execute: the plan's default kernel
                torch.cuda.synchronize()
                times = []
                for _ in range(20):
                    ev[0].record(stream)
                    pl2.execute(1.0, 0.0, prec, 1)
                    ev[1].record(stream)
                    torch.cuda.synchronize()
                    times.append(ev[0].elapsed_time(ev[1]))
                t = statistics.median(times)
                extras[name] = {"numeric_gflops": flops / (t * 1e-3) / 1e9, "ms": t,
                                "speedup_vs_fp64_numeric": num_avg / t,
                                "first_execute_ms": min(first), "repeats_timed": len(times),
                                "note": "median of 20 repeat executes of one plan after 3 "
                                        "(slicing of the current data + products); "
                                        "first_execute_ms: a fresh plan's first execute"}
                if prec == bst.BST_FP64_EMU_BF16:
                    c = bst.bst_plan_emu_costs(pl2.handle)
                    extras[name]["kernel"] = "k_pan_mma (tcgen05 panels)" if c["panel"] else \
                        "k_num_emu_bf16_persist1 (mma.sync C blocks)"
                    extras[name]["roofline"] = emu_roofline([pl2], t, bst.context(local_rank))
                if sample is not None:
                    extras[name]["rel_err_vs_oracle_sample"] = sample.error(pl2)
                del pl, pl2
            except bst.BstError as e:
                extras[name] = {"unavailable": e.name}
        if sample is not None:
            extras["error_sample"] = sample.describe()
        line["precision_variants"] = extras
        line["fp64_stacks_13_23"] = single_stacks(local_rank, stream)
        if rank == 0 and not args.no_configs:
            line["other_configs"] = other_configs(local_rank, stream)

    if rank == 0 and world == 1 and not args.no_cpu:
        rows = CPU_SAMPLE_ROWS if args.nb == 4000 else (args.nb // 4, 3 * args.nb // 4)
        fl, times = cpu_baseline(p, rows, steps=1)
        line["cpu_baseline"] = {
            "value": fl / times[0] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"block rows {rows[0]}..{rows[1]} of A times all of B "
                      f"({fl:.3e} flop, {times[0]:.1f} s, single thread)"}
        if not args.no_cpu_parallel:
            ncores = min(len(os.sched_getaffinity(0)), 64)
            flp, tp = cpu_baseline_parallel(rank_seed(rank), args.nb, (0, args.nb), ncores)
            line["cpu_baseline_parallel"] = {
                "value": flp / tp / 1e9, "unit": UNIT, "cores": ncores, "kind": "oracle",
                "sample": f"all {args.nb} block rows of A times B, one process per core over "
                          f"disjoint block rows ({flp:.3e} flop, {tp:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def single_stacks(local_rank, stream, nb=1000):
    """Native FP64 numeric throughput and roofline fraction on single-stack versions of
    the banded workload: every (m, n, k) in {13, 23}^3, same band and filter."""
    import torch

    from paper_1910_13555_gb300 import bst
    from paper_1910_13555_gb300.workloads import banded
    out = []
    for m in (13, 23):
        for n in (13, 23):
            for k in (13, 23):
                p = banded(seed=1102, nb=nb, block_mkn=(m, k, n))
                mk = lambda x: bst.Matrix.from_host(x.row_sizes, x.col_sizes, x.rows, x.cols,
                                                    x.data, device=local_rank)
                A, B = mk(p.A), mk(p.B)
                plan = bst.multiply_plan(A, B, None, p.eps, device=local_rank)
                plan.alloc_result(local_rank)
                plan.execute(1.0, 0.0, bst.BST_FP64, 1)
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                times = []
                for _ in range(3):
                    ev[0].record(stream)
                    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
                    ev[1].record(stream)
                    torch.cuda.synchronize()
                    times.append(ev[0].elapsed_time(ev[1]))
                t = statistics.median(times)
                f = plan.stats()["flops"]
                out.append({"mnk": [m, n, k], "flop": f, "ms": t,
                            "gflops": f / (t * 1e-3) / 1e9,
                            "frac": f / (t * 1e-3) / 1e12 / FP64_PEAK_TFLOPS})
                del plan, A, B
    tot_f = sum(o["flop"] for o in out)
    tot_t = sum(o["ms"] for o in out)
    return {"workload": f"banded {nb}x{nb} blocks, one (m, n, k) per run", "stacks": out,
            "aggregate_frac": tot_f / (tot_t * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}


def _median_ms(fn, stream, reps=20, warmup=3):
    """Median of `reps` CUDA-event-timed runs of fn on `stream` after `warmup` runs."""
    import torch
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    return statistics.median(times)


def _rel(got, ref):
    import numpy as np
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def _gather(data, offs, lens):
    import numpy as np
    import torch
    idx = np.concatenate([np.arange(o, o + n) for o, n in zip(offs, lens)])
    return data[torch.as_tensor(idx, device=data.device)].cpu().numpy()


def _sample_err_matrix(p, plan, row_sizes, col_sizes, nsample=32, seed=0):
    """Relative error of a product on sampled C blocks (the oracle computes exactly those)."""
    import numpy as np

    import oracle
    rows, cols, offs = plan.result.index()
    if len(rows) == 0:
        return 0.0
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(rows), min(nsample, len(rows)), replace=False))
    ref, _ = oracle.multiply_sample(p.A, p.B, p.C_in, p.alpha, p.beta, p.eps, rows[sel], cols[sel],
                                    transa=p.transa, transb=p.transb, row_sizes=row_sizes,
                                    col_sizes=col_sizes)
    lens = row_sizes[rows[sel]].astype(np.int64) * col_sizes[cols[sel]]
    return _rel(_gather(plan.result.data, offs[sel], lens), ref)


def ksplit_simulated(p, nproc, whole, local_rank, stream):
    """The K-split product of a tall-skinny workload with `nproc` processes run one after
    another on one GPU: median times of all partial multiplies and of all owner sums
    (CUDA events, 20 after 3 warm-ups), the owner-sum kernel's HBM roofline (bytes read
    and written by bst_sum_parts over its time) and the error against the undivided
    product `whole` (device data in its C layout)."""
    import numpy as np
    import torch

    from paper_1910_13555_gb300 import bst, ksplit
    A, B = p.A, p.B
    ka = ksplit.k_index(A.rows, A.cols, p.transa, "A")
    kb = ksplit.k_index(B.rows, B.cols, p.transb, "B")
    ea = A.row_sizes[A.rows].astype(np.int64) * A.col_sizes[A.cols]
    eb = B.row_sizes[B.rows].astype(np.int64) * B.col_sizes[B.cols]
    r = ksplit.k_ranges(ka, ea, kb, eb, A.row_sizes if p.transa == "T" else A.col_sizes, nproc)
    plans, mats, pats = [], [], []
    for i in range(nproc):
        ra, ca, da = ksplit.select_k_range(A.row_sizes, A.col_sizes, A.rows, A.cols, A.data,
                                           p.transa, "A", r[i], r[i + 1])
        rb, cb, db = ksplit.select_k_range(B.row_sizes, B.col_sizes, B.rows, B.cols, B.data,
                                           p.transb, "B", r[i], r[i + 1])
        Ai = bst.Matrix.from_host(A.row_sizes, A.col_sizes, ra, ca, da, device=local_rank)
        Bi = bst.Matrix.from_host(B.row_sizes, B.col_sizes, rb, cb, db, device=local_rank)
        pl = bst.multiply_plan(Ai, Bi, None, p.eps, p.transa, p.transb, device=local_rank)
        pl.alloc_result(local_rank)
        plans.append(pl)
        mats.append((Ai, Bi))
    f = sum(pl.stats()["flops"] for pl in plans)

    def partials():
        for pl in plans:
            pl.execute(1.0, 0.0, bst.BST_FP64, 1)
    ms_part = _median_ms(partials, stream)
    parts = []
    for pl in plans:
        rows, cols, _ = pl.result.index()
        pats.append((rows, cols))
        parts.append(pl.result.data[:pl.result.info[3]])
    rs = A.col_sizes if p.transa == "T" else A.row_sizes
    cs = B.row_sizes if p.transb == "T" else B.col_sizes
    lay = ksplit.exchange_layout(pats, rs, cs)
    dev = torch.device("cuda", local_rank)
    bufs, tabs, outs, nbytes = [], [], [], 0
    for q in range(nproc):
        chunks = [parts[i][int(lay.send[i, :q].sum()):int(lay.send[i, :q + 1].sum())]
                  for i in range(nproc)]
        bufs.append(torch.cat(chunks))
        _, _, offs = lay.owned(q)
        tabs.append((torch.as_tensor(np.ascontiguousarray(offs, np.int64)).to(dev),
                     torch.as_tensor(np.ascontiguousarray(lay.src_off[q], np.int64)).to(dev)))
        outs.append(torch.empty(int(offs[-1]), dtype=torch.float64, device=dev))
        nbytes += 8 * (bufs[-1].numel() + int(offs[-1]))

    def sums():
        for q in range(nproc):
            n = len(tabs[q][0]) - 1
            if n:
                bst.bst_sum_parts(bst.context(local_rank), nproc, n, tabs[q][0], tabs[q][1],
                                  bufs[q], outs[q])
    # the owners' sums replayed from a CUDA graph: one launch each, back to back on the
    # device, so the time is the kernels' and not the host's launch overhead
    sums()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cs):
        sums()
    ms_sum = _median_ms(g.replay, stream)
    got = torch.cat(outs)
    err = float(torch.linalg.norm(got - whole) / torch.linalg.norm(whole))
    achieved = nbytes / (ms_sum * 1e-3) / 1e9
    return {"processes": nproc, "k_ranges": [int(x) for x in r], "flop": f,
            "partials_ms": ms_part, "partials_gflops": f / (ms_part * 1e-3) / 1e9,
            "sum_ms": ms_sum, "sum_bytes": nbytes,
            "sum_roofline": {"bound": "hbm", "kernel": "k_sum_parts", "achieved": achieved,
                             "peak": MEASURED_HBM_GBS, "unit": "GB/s",
                             "frac": achieved / MEASURED_HBM_GBS if MEASURED_HBM_GBS else None},
            "rel_err_vs_undivided": err,
            "note": "processes simulated one after another on one GPU; the owners' sums "
                    "timed as one graph replay; the all-to-all between partial products and "
                    "owners is not timed"}


def other_configs(local_rank, stream):
    """The other workloads of the method, measured like the headline: numeric GFLOP/s
    (CUDA events, median of 20 after 3 warm-ups), fraction of the FP64 unit-count peak
    (native rows) or the emulated path's own roofline (emulated rows), and error against
    the CPU oracle on sampled output blocks."""
    import numpy as np
    import torch

    import oracle
    from paper_1910_13555_gb300 import bst
    from paper_1910_13555_gb300.workloads import (batched, plain, rank3, rank4, rect_case2,
                                                  tall_skinny)

    def mk(m):
        return bst.Matrix.from_host(m.row_sizes, m.col_sizes, m.rows, m.cols, m.data,
                                    device=local_rank)

    def rate(f, ms):
        return {"gflops": f / (ms * 1e-3) / 1e9, "ms": ms,
                "frac": f / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}

    def rate_emu(f, ms, plans):
        """Emulated FP64: credited GFLOP/s, the ratio of that rate to the FP64 peak (a
        speedup measure, not a roofline fraction) and the roofline fraction of the
        emulated path itself (emu_roofline)."""
        return {"gflops": f / (ms * 1e-3) / 1e9, "ms": ms,
                "credited_over_fp64_peak": f / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                "roofline": emu_roofline(plans, ms, bst.context(local_rank))}

    out = {}
    # 40 x 40 blocks of size 5, 10 % occupancy, no filter
    p = plain()
    A, B = mk(p.A), mk(p.B)
    plan = bst.multiply_plan(A, B, None, 0.0, device=local_rank)
    plan.alloc_result(local_rank)
    ms = _median_ms(lambda: plan.execute(1.0, 0.0, bst.BST_FP64, 1), stream)
    ref = oracle.multiply(p.A, p.B)
    n = plan.result.info[3]
    out["plain_40x40_size5"] = dict(rate(plan.stats()["flops"], ms),
                                    rel_err_vs_oracle=_rel(plan.result.data[:n].cpu().numpy(),
                                                           ref["data"]))
    # the no-allocation execute (CTA-level K split into the static array), split 2
    ms = _median_ms(lambda: bst.bst_multiply_execute_static(plan.handle, 1.0, 0.0, 2), stream)
    out["plain_40x40_size5"]["static_split_2"] = dict(
        rate(plan.stats()["flops"], ms),
        rel_err_vs_oracle=_rel(plan.result.data[:n].cpu().numpy(), ref["data"]))
    del plan, A, B
    # tall-skinny C = A^T B (100000 x 400 blocks), split-K
    p = tall_skinny()
    A, B = mk(p.A), mk(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, "T", "N", device=local_rank)
    plan.alloc_result(local_rank)
    f = plan.stats()["flops"]
    ts = {}
    # split 1 and the automatic choice run the staged kernel; split 4 the CTA-level K
    # split (k_num_fp64 into 4 partial copies of C, then k_splitk_reduce)
    for split in (1, 0, 4):
        ms = _median_ms(lambda: plan.execute(1.0, 0.0, bst.BST_FP64, split), stream)
        ts[f"split_{split or 'auto'}"] = dict(rate(f, ms), split_k=plan.stats()["split_k"],
                                              rel_err_vs_oracle_sample=_sample_err_matrix(
                                                  p, plan, p.A.col_sizes, p.B.col_sizes))
    ms = _median_ms(lambda: plan.execute(1.0, 0.0, bst.BST_FP64_EMU_BF16, 1), stream)
    ts["emu_bf16"] = dict(rate_emu(f, ms, [plan]), rel_err_vs_oracle_sample=_sample_err_matrix(
        p, plan, p.A.col_sizes, p.B.col_sizes))
    # the K split of the same product over 4 processes (paper Sec. 3.1), the processes
    # simulated one after another on this GPU: partial products, then every owner's
    # fixed-order sum (bst_sum_parts); the all-to-all between them is not timed here
    plan.execute(1.0, 0.0, bst.BST_FP64, 1)
    torch.cuda.synchronize()
    whole = plan.result.data[:plan.result.info[3]].clone()
    ts["ksplit_4_simulated"] = ksplit_simulated(p, 4, whole, local_rank, stream)
    out["tall_skinny_AtB"] = ts
    del plan, A, B, whole
    # the same shape with a small C (40 x 40 blocks, 1600 tiles for about 1800 resident
    # warps): the case the K split is for
    p = tall_skinny(nmn=40, window=40)
    A, B = mk(p.A), mk(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, "T", "N", device=local_rank)
    plan.alloc_result(local_rank)
    f = plan.stats()["flops"]
    sc = {"flop": f, "c_blocks": plan.stats()["n_c_blocks"]}
    for split in (1, 2, 4, 8, 0):
        ms = _median_ms(lambda: plan.execute(1.0, 0.0, bst.BST_FP64, split), stream)
        sc[f"split_{split or 'auto'}"] = dict(rate(f, ms), split_k=plan.stats()["split_k"],
                                              rel_err_vs_oracle_sample=_sample_err_matrix(
                                                  p, plan, p.A.col_sizes, p.B.col_sizes))
    out["tall_skinny_small_C"] = sc
    del plan, A, B
    # 64 independent products in one persistent launch, replayed from a CUDA graph
    probs = batched()
    mats, plans = [], []
    for q in probs:
        A, B = mk(q.A), mk(q.B)
        pl = bst.multiply_plan(A, B, None, q.eps, device=local_rank)
        pl.alloc_result(local_rank)
        mats.append((A, B))
        plans.append(pl)
    f = sum(pl.stats()["flops"] for pl in plans)
    ones, zeros = np.ones(len(plans)), np.zeros(len(plans))
    # error over all of C on the four smallest problems (the oracle computes them whole)
    small = sorted(range(len(plans)), key=lambda q: plans[q].stats()["flops"])[:4]
    refs = {q: oracle.multiply(probs[q].A, probs[q].B, None, 1.0, 0.0, probs[q].eps)["data"]
            for q in small}
    ctx = bst.context(local_rank)
    old_pan = bst.bst_tune_get(ctx, bst.BST_TUNE_EMU_PANEL)
    bt = {}
    # emulated rows: the default (every plan on the tcgen05 panel kernel) and the
    # C-block kernel with row-scaled digits
    for name, prec, pan in (("fp64", bst.BST_FP64, old_pan),
                            ("emu_bf16", bst.BST_FP64_EMU_BF16, old_pan),
                            ("emu_bf16_c_block_kernel", bst.BST_FP64_EMU_BF16, 0)):
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_PANEL, pan)
        batch = bst.bst_batch_create(ctx, [pl.handle for pl in plans])
        bst.bst_batch_execute(batch, ones, zeros, prec)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=cs):
            bst.bst_batch_execute(batch, ones, zeros, prec, stream=cs)
        ms = _median_ms(g.replay, stream)
        full = max(_rel(plans[q].result.data[:plans[q].result.info[3]].cpu().numpy(), refs[q])
                   for q in small)
        blk = max(_sample_err_matrix(probs[q], plans[q], probs[q].A.row_sizes,
                                     probs[q].B.col_sizes, nsample=8, seed=q)
                  for q in (0, 7, 31, 63))
        row = dict(rate(f, ms) if prec == bst.BST_FP64 else rate_emu(f, ms, plans),
                   rel_err_vs_oracle=full,
                   max_rel_err_of_sampled_blocks=blk,
                   launch="one persistent kernel per replay (CUDA graph)")
        if prec != bst.BST_FP64:
            row["plans_on_panel_kernel"] = int(sum(
                bst.bst_plan_emu_costs(pl.handle)["panel"] for pl in plans)) if pan else 0
        bt[name] = row
        del g
        bst.bst_batch_destroy(batch)
    bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_PANEL, old_pan)
    out["batched_64"] = dict(bt, flop=f,
                             error_note="rel_err_vs_oracle: relative Frobenius error over all "
                                        "of C, worst of the 4 smallest problems; sampled "
                                        "blocks: 8 C blocks of each of 4 problems, each set "
                                        "measured on its own (block scales span 8 decades)")
    del plans, mats
    # rank-3 contraction R(mu,lam) = sum_{P,nu} T(P,mu,nu) U(P,nu,lam), forward + adjoint
    w = rank3()
    t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data, device=local_rank)
    t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data, device=local_rank)
    cplan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, device=local_rank)
    torch.cuda.synchronize()
    f = cplan.stats()["flops"]
    R = cplan.result
    ms = _median_ms(lambda: cplan.execute(1.0, 0.0, bst.BST_FP64, 1), stream)
    idx, offs = R.index()
    rs = [w.T1.block_sizes[1], w.T2.block_sizes[2]]
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(len(idx), min(32, len(idx)), replace=False))
    ref, _ = oracle.contract_sample(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order, None,
                                    1.0, 0.0, 0.0, idx[sel], rs)
    lens = rs[0][idx[sel, 0]].astype(np.int64) * rs[1][idx[sel, 1]]
    fwd = dict(rate(f, ms), rel_err_vs_oracle_sample=_rel(_gather(R.data, offs[sel], lens), ref))
    ne = R.info[2]
    dR = R.data[:ne].clone()
    dT = torch.empty_like(t1.data)
    dU = torch.empty_like(t2.data)
    ms_adj = _median_ms(lambda: bst.bst_plan_adjoint(cplan.handle, dR, dT, dU, None, 1.0, 0.0),
                        stream)
    fwd["slab_read"] = cplan.schedule_info()["slab"]
    del cplan, R
    # the same forward through the other remap of T(P, mu, nu): its blocks permuted into
    # a (mu, P, nu) copy before every execute, instead of read in place as P slabs
    ctx = bst.context(local_rank)
    prev = bst.bst_tune_get(ctx, bst.BST_TUNE_CONTRACT_SLAB)
    bst.bst_tune_set(ctx, bst.BST_TUNE_CONTRACT_SLAB, 0)
    splan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, device=local_rank)
    bst.bst_tune_set(ctx, bst.BST_TUNE_CONTRACT_SLAB, prev)
    torch.cuda.synchronize()
    ms_s = _median_ms(lambda: splan.execute(1.0, 0.0, bst.BST_FP64, 1), stream)
    R = splan.result
    fwd_s = dict(rate(f, ms_s), slab_read=splan.schedule_info()["slab"],
                 rel_err_vs_oracle_sample=_rel(_gather(R.data, offs[sel], lens), ref))
    out["rank3_contraction"] = {"forward": fwd, "forward_permuted_copy": fwd_s,
                                "adjoint": dict(rate(2.0 * f, ms_adj),
                                                note="dT and dU, 2x the forward flop")}
    del splan, t1, t2, R, dR, dT, dU
    # rectangular case S_B << S_A, S_C: C = A B with a small B
    p = rect_case2()
    A, B = mk(p.A), mk(p.B)
    plan = bst.multiply_plan(A, B, None, p.eps, device=local_rank)
    plan.alloc_result(local_rank)
    f = plan.stats()["flops"]
    rc = {}
    for name, prec in (("fp64", bst.BST_FP64), ("emu_bf16", bst.BST_FP64_EMU_BF16)):
        ms = _median_ms(lambda: plan.execute(1.0, 0.0, prec, 1), stream)
        rc[name] = dict(rate(f, ms) if prec == bst.BST_FP64 else rate_emu(f, ms, [plan]),
                        rel_err_vs_oracle_sample=_sample_err_matrix(
            p, plan, p.A.row_sizes, p.B.col_sizes))
    out["rect_case2_small_B"] = dict(rc, flop=f)
    del plan, A, B
    # rank-4 x rank-3 over two index pairs, permuted view, reordered result
    w = rank4()
    t1 = bst.Tensor.from_host(w.T1.block_sizes, w.T1.index, w.T1.data, device=local_rank)
    t2 = bst.Tensor.from_host(w.T2.block_sizes, w.T2.index, w.T2.data, device=local_rank)
    cplan = bst.contract(t1, t2, w.c1, w.c2, w.f1, w.f2, w.result_order, device=local_rank)
    torch.cuda.synchronize()
    f = cplan.stats()["flops"]
    R = cplan.result
    ms = _median_ms(lambda: cplan.execute(1.0, 0.0, bst.BST_FP64, 1), stream)
    idx, offs = R.index()
    rs = [w.T1.block_sizes[1], w.T2.block_sizes[2], w.T1.block_sizes[3]]
    sel = np.sort(np.random.default_rng(2).choice(len(idx), min(32, len(idx)), replace=False))
    ref, _ = oracle.contract_sample(w.T1, w.T2, w.c1, w.c2, w.f1, w.f2, w.result_order, None,
                                    1.0, 0.0, 0.0, idx[sel], rs)
    lens = np.ones(len(sel), np.int64)
    for d in range(3):
        lens *= rs[d][idx[sel, d]].astype(np.int64)
    fwd4 = dict(rate(f, ms), rel_err_vs_oracle_sample=_rel(_gather(R.data, offs[sel], lens), ref))
    ne = R.info[2]
    dR = R.data[:ne].clone()
    dV = torch.empty_like(t1.data)
    dU = torch.empty_like(t2.data)
    ms_adj = _median_ms(lambda: bst.bst_plan_adjoint(cplan.handle, dR, dV, dU, None, 1.0, 0.0),
                        stream)
    out["rank4_contraction"] = dict(fwd4, adjoint=dict(rate(2.0 * f, ms_adj),
                                                       note="dV and dU, 2x the forward flop"))
    del cplan, R, dR, dV, dU, t1, t2
    return out


def e2e_leg(p, local_rank, steps, stream, barrier, world, dev):
    """The same metric through the public API from host buffers: each step copies A's
    and B's data from pinned host memory (H2D), creates the matrices from the host index
    arrays, plans, executes and reads all of C_out back into pinned host memory (D2H).
    Steps alternate between two compute streams, and each step's D2H runs on copy
    streams of its own (the read-back in D2H_SPLIT parts) that wait for the execute, so
    one step's D2H overlaps the next steps' uploads, plans and executes (on one stream,
    the next upload two steps later queued behind the 4 GB read-back and the SMs waited
    for it), as a caller streaming independent products would run them."""
    import torch

    from paper_1910_13555_gb300 import bst

    ha = torch.from_numpy(p.A.data).pin_memory()
    hb = torch.from_numpy(p.B.data).pin_memory()
    ctx = bst.context(local_rank)
    streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    # the read-back of C in D2H_SPLIT parts, each on a copy stream of its own, so that
    # several copy engines move it at once
    copies = [[torch.cuda.Stream(device=dev) for _ in range(D2H_SPLIT)] for _ in range(2)]
    hcs = [None, None]
    alive = [None, None]  # objects of the step in flight on each stream
    info = {"flops": 0.0, "n": 0}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    marks = []  # per step: events after H2D, after create + plan, after execute, D2H start / end

    def one(i):
        slot = i % 2
        s = streams[slot]
        m = [ev() for _ in range(5 + D2H_SPLIT)]
        with torch.cuda.stream(s):
            sh = s.cuda_stream
            m[0].record(s)
            da = ha.to(dev, non_blocking=True)
            db = hb.to(dev, non_blocking=True)
            m[1].record(s)
            A = bst.Matrix(bst.bst_matrix_create(ctx, p.A.row_sizes, p.A.col_sizes, p.A.rows,
                                                 p.A.cols, da, stream=sh), da)
            B = bst.Matrix(bst.bst_matrix_create(ctx, p.B.row_sizes, p.B.col_sizes, p.B.rows,
                                                 p.B.cols, db, stream=sh), db)
            plan = bst.multiply_plan(A, B, None, p.eps, device=local_rank, stream=sh)
            plan.alloc_result(local_rank)
            m[2].record(s)
            plan.execute(1.0, 0.0, bst.BST_FP64, 1, stream=sh)
            m[3].record(s)
            n = plan.result.info[3]
            if hcs[slot] is None or hcs[slot].numel() < n:
                hcs[slot] = torch.empty(n, dtype=torch.float64).pin_memory()
        cut = [n * j // D2H_SPLIT for j in range(D2H_SPLIT + 1)]
        for j, cs in enumerate(copies[slot]):
            cs.wait_event(m[3])
            with torch.cuda.stream(cs):
                if j == 0:
                    m[4].record(cs)
                plan.result.data.record_stream(cs)
                hcs[slot][cut[j]:cut[j + 1]].copy_(plan.result.data[cut[j]:cut[j + 1]],
                                                   non_blocking=True)
                m[5 + j].record(cs)
        alive[slot] = (plan, A, B, da, db)
        info["flops"] = plan.stats()["flops"]
        info["n"] = n
        return m

    one(0)
    one(1)
    torch.cuda.synchronize()
    barrier()
    t = time.perf_counter()
    for i in range(steps):
        marks.append(one(i))
    torch.cuda.synchronize()
    barrier()
    dt = (time.perf_counter() - t) / steps
    alive[0] = alive[1] = None
    flops = info["flops"]
    dt, flops = reduce_over_ranks(dt, flops, world, dev)
    h2d = (p.A.data.nbytes + p.B.data.nbytes + 8 * (p.A.nblocks + p.B.nblocks) +
           4 * (len(p.A.row_sizes) + len(p.A.col_sizes) + len(p.B.row_sizes) + len(p.B.col_sizes)))
    phase = lambda a, b: statistics.median(x[a].elapsed_time(x[b]) for x in marks)
    d2h = statistics.median(max(x[4].elapsed_time(x[5 + j]) for j in range(D2H_SPLIT))
                            for x in marks)
    return {"value": flops / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(8 * info["n"]), "ms_per_step": dt * 1e3,
            "steps_timed": steps,
            "streams": f"2 compute + 2 x {D2H_SPLIT} copy (the read-back in {D2H_SPLIT} parts)",
            "phases_ms_median": {"h2d": phase(0, 1), "create_and_plan": phase(1, 2),
                                 "execute": phase(2, 3), "d2h": d2h},
            "phases_note": "CUDA events per step on its own streams; phases of consecutive "
                           "steps overlap (the read-back of one step runs beside the next "
                           "steps' uploads, plans and executes), so they do not add up to "
                           "ms_per_step"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
