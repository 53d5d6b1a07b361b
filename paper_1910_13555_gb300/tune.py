"""Autotuner of the library's kernel choices (bst_tune_set), written for this library.

What it tunes, per (m, n) C block class:
* the thread mapping of the emulated-FP64 tensor-core kernel -- whether the 16-row MMA
  tiles run over the C block's rows (0) or over its columns (1, computing
  C^T = op(B)^T op(A)^T on the same digit planes).  The two mappings use different
  numbers of 16 x 8 tiles and load the two operands' fragments in different
  proportions, so which one is faster depends on m, n and the inner sizes k;
* the largest inner split of the native-FP64 staged kernel's tiles: a tile whose m n
  outputs leave lanes idle (5 x 13 = 65 outputs on 3 x 32 lanes) can spread its inner
  dimension over s lane groups and add the s partial sums at the end.  The library picks
  s per tile by counting FP64 instructions; the tuner bounds it per class by timing.
For every class present in a plan the tuner times the plan's execute with that class set
to each choice (the others unchanged), keeps the fastest, and returns a table that can be
saved as JSON (keyed by GPU name) and applied to a context later.

Per contraction, tune_contract_slab chooses between the two remaps of a first tensor
stored as (outer contracted, free, inner contracted) modes: a permuted copy before every
execute, or reading each block in place as consecutive contiguous slabs.

Timing uses CUDA events on the current stream, after a warm-up, minimum over repeats.
"""
from __future__ import annotations

import json
import os

from . import bst


def plan_classes(plan) -> list:
    """Distinct (m, n) C block classes of a plan's stacks (from its (m, n, k) buckets)."""
    st = bst.bst_plan_get_stacks(plan.handle)
    return sorted({(int(m), int(n)) for m, n, _ in st["mnk"].tolist()})


def time_execute(plan, precision, reps=3, warmup=1) -> float:
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.execute(1.0, 0.0, precision, 1)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        plan.execute(1.0, 0.0, precision, 1)
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_emulated(plan, device=0, reps=3) -> dict:
    """Choose the emulated-FP64 tile mapping per (m, n) class of `plan` (which must have
    its result bound) and leave the choices set in the context.  Returns
    {(m, n): {"swap": best, "ms": {0: t0, 1: t1}}}."""
    ctx = bst.context(device)
    table = {}
    for (m, n) in plan_classes(plan):
        times = {}
        for v in (0, 1):
            bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_SWAP, v, m, n)
            times[v] = time_execute(plan, bst.BST_FP64_EMU_BF16, reps)
        best = min(times, key=times.get)
        bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_SWAP, best, m, n)
        table[(m, n)] = {"swap": best, "ms": times}
    return table


SPLIT_CHOICES = (1, 2, 4, 16)  # largest split tried per class (16: the built-in bound)


def tune_fp64_split(plan, device=0, reps=3, choices=SPLIT_CHOICES) -> dict:
    """Choose the largest inner split of the native-FP64 staged kernel per (m, n) class
    of `plan` (result bound) and leave the choices set in the context.  Returns
    {(m, n): {"split": best, "ms": {choice: t}}}."""
    ctx = bst.context(device)
    table = {}
    for (m, n) in plan_classes(plan):
        times = {}
        for v in choices:
            bst.bst_tune_set(ctx, bst.BST_TUNE_F64_SPLIT, v, m, n)
            times[v] = time_execute(plan, bst.BST_FP64, reps)
        best = min(times, key=times.get)
        bst.bst_tune_set(ctx, bst.BST_TUNE_F64_SPLIT, best, m, n)
        table[(m, n)] = {"split": best, "ms": times}
    return table


def tune_contract_slab(T1, T2, c1, c2, f1, f2, result_order=None, R_in=None, eps=0.0, device=0,
                       reps=3) -> dict:
    """Choose how a contraction reads a first tensor stored (outer contracted, free, inner
    contracted): in place as slabs (1) or through a permuted copy (0).  Builds the plan
    both ways, times its native-FP64 execute, leaves the faster choice set in the context
    (BST_TUNE_CONTRACT_SLAB, taken by plans created afterwards).  Returns
    {"slab": best, "ms": {0: t0, 1: t1}, "eligible": {0: ..., 1: ...}} where eligible says
    whether the plan really read slabs."""
    ctx = bst.context(device)
    times, used = {}, {}
    for v in (0, 1):
        bst.bst_tune_set(ctx, bst.BST_TUNE_CONTRACT_SLAB, v)
        plan = bst.contract_plan(T1, T2, c1, c2, f1, f2, result_order, R_in, eps, device)
        plan.alloc_result(device)
        times[v] = time_execute(plan, bst.BST_FP64, reps)
        used[v] = plan.schedule_info()["slab"] == bool(v)
        del plan
    best = min(times, key=times.get)
    bst.bst_tune_set(ctx, bst.BST_TUNE_CONTRACT_SLAB, best)
    return {"slab": best, "ms": times, "eligible": used}


def gpu_name(device=0) -> str:
    import torch
    return torch.cuda.get_device_name(device)


_CHOICE_KEYS = ("swap", "split")


def table_to_json(table: dict, gpu: str) -> dict:
    """Entries carry "swap" (emulated-FP64 mapping) and/or "split" (native-FP64 bound)."""
    return {"gpu": gpu, "entries": [
        dict({"m": m, "n": n, "ms": v.get("ms", {})},
             **{k: int(v[k]) for k in _CHOICE_KEYS if k in v})
        for (m, n), v in sorted(table.items())]}


def table_from_json(doc: dict) -> dict:
    return {(int(e["m"]), int(e["n"])): dict({"ms": e.get("ms", {})},
                                             **{k: int(e[k]) for k in _CHOICE_KEYS if k in e})
            for e in doc["entries"]}


def merge_tables(*tables: dict) -> dict:
    """One table from several (e.g. tune_emulated's and tune_fp64_split's)."""
    out = {}
    for t in tables:
        for key, v in t.items():
            e = out.setdefault(key, {"ms": {}})
            for k in _CHOICE_KEYS:
                if k in v:
                    e[k] = v[k]
                    e["ms"] = dict(e["ms"], **{f"{k}={c}": t_ for c, t_ in v["ms"].items()})
    return out


def save_table(table: dict, path: str, gpu: str) -> None:
    """Write (or update the `gpu` entry of) a JSON tune file."""
    docs = {}
    if os.path.exists(path):
        with open(path) as f:
            docs = json.load(f)
    docs[gpu] = table_to_json(table, gpu)
    with open(path, "w") as f:
        json.dump(docs, f, indent=1, default=str)


def apply_table(table: dict, device=0) -> None:
    ctx = bst.context(device)
    for (m, n), v in table.items():
        if "swap" in v:
            bst.bst_tune_set(ctx, bst.BST_TUNE_EMU_SWAP, int(v["swap"]), m, n)
        if "split" in v:
            bst.bst_tune_set(ctx, bst.BST_TUNE_F64_SPLIT, int(v["split"]), m, n)


def load_table(path: str, gpu: str, device=0) -> dict:
    """Apply the saved choices for `gpu` to the context; {} when the file has none."""
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        docs = json.load(f)
    if gpu not in docs:
        return {}
    table = table_from_json(docs[gpu])
    apply_table(table, device)
    return table
