"""The benchmark's N-rank path on the CPU with two gloo ranks: each rank works on its own
problem (different seeds, no data-path collective), the whole-job time is the slowest
rank's and the work is summed; under torchrun the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, local_rank, world = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
flops = 1.0e9 * (rank + 1)
out = bench.reduce_over_ranks(ms, flops, world, "cpu")
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "seed": bench.rank_seed(rank), "ms": out[0], "flops": out[1]}}))
"""


def _launch(code, world=2, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_two_gloo_ranks_reduce_time_and_work():
    outs = _launch(_WORKER.format(root=ROOT))
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["ms"] == 15.0                 # the slowest rank's time
        assert r["flops"] == 3.0e9             # the work of both ranks
    assert res[0]["seed"] != res[1]["seed"]    # independent problems


def test_reference_arm_runs_on_rank_zero_only():
    pytest.importorskip("numpy")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            "sys.argv = ['bench.py', '--impl', 'reference', '--gpus', '2', '--steps', '1', "
            "'--warmup', '0']; sys.exit(bench.main())")
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""              # rank 1 prints nothing and does no work
