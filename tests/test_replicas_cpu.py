"""The multi-process path of bench.py on CPU (gloo, world size 2).

The sort does not shard (an LSD pass scatters across the whole array), so N
processes run N independent replicas: each rank sorts its own array, the
time is the maximum over ranks, and the value counts every rank's items.
These tests run that host logic with two gloo ranks and no GPU.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1008_2849_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Rank r reports a local time of 10 * (r + 1) ms: all must agree on the max.
        local_ms = 10.0 * (rank + 1)
        dist.barrier()
        worst = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        value = bench.job_throughput(world, 4, 1000, worst / 1e3)
        # Every rank's replica input is its own array.
        k = inputs.keys("uniform", 4096, seed=bench.replica_seed(rank))
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"worst": worst, "value": value, "head": k[:8].tolist()}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["worst"] == 20.0                 # the slowest rank's time
        assert r["value"] == world * 4 * 1000 / 0.020
    assert res[0]["head"] != res[1]["head"]       # independent replicas


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench.job_throughput(1, 10, 1 << 28, 2.0) == 10 * (1 << 28) / 2.0
    assert bench.replica_seed(0) == bench.KEY_SEED


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched as two ranks: rank 0 alone times
    the oracle and prints the JSON line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "2", "--warmup", "3", "--reference-sample-log2", "18"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(s) for s in p.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["unit"] == "pairs/s"
    assert line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert np.isfinite(line["ms_per_step"])
