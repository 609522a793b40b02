"""Benchmark of the GB300 radix sort.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete sort (digit histograms, prefix/plan, four scatter
passes) of 2^28 (uint32 key, uint32 value = index) pairs with uniform keys
(seed 2), through the C ABI call rs_sort_pairs_ex on the current stream.
Every step sorts its own freshly copied input (2 GiB, far larger than the
129 MB L2), so no step sees data left in cache by the previous one.

On one GPU the line also carries the metric's other parts, from legs run
after the timed region (bench_extras): the latency of a 2^20-key sort, the
batched segmented sort of 4096 arrays (2^28 pairs) against a loop of
per-array sorts, and the serving loop's p50/p99 latency against serial plain
sorts, each with its own clock samples.

Printed (rank 0, one JSON line): pairs/s for the whole job; the dominant
kernel's achieved HBM bandwidth against the measured copy peak (roofline);
the same metric end to end through rs_sort_pairs_host_batch with pinned host
buffers (every step's upload and download included, overlapping the sorts of
neighbouring steps), next to one rs_sort_pairs_host call per array; the CPU
oracle's throughput on a bounded sample (cpu_baseline); SM clocks sampled
during the timed region.

With N > 1 (torchrun) the ranks sort ONE array of N * 2^28 pairs held in
shards, by Alg. 2's partition (--mode partition, the default there): every
rank partitions its shard by the top byte, the bucket sizes are gathered,
the items are exchanged by contiguous top-byte ranges balanced by count
(NCCL all-to-all), and every rank sorts what it received.  --mode sort runs
N independent replicas instead.  Either way the time is the maximum over
ranks and the value counts all ranks' pairs.

--impl reference times the CPU oracle (the plain LSD counting sort of the
paper's Sec. 3/4, run on all host cores) on a bounded sample of the same
workload; there is no GPU in that arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1008_2849_gb300 import inputs, roofline  # noqa: E402

METRIC = "32-bit key-value pairs sorted/s"
UNIT = "pairs/s"
N_PAIRS = 1 << 28
KEY_SEED = 2
WORKLOAD = "sort_pairs_u32_2^28_uniform"
ONESWEEP_SOURCES = ("paper_1008_2849_gb300/csrc/rs_onesweep.cuh",
                    "paper_1008_2849_gb300/csrc/rs_onesweep_launch.cuh",
                    "paper_1008_2849_gb300/csrc/rs_device.cuh",
                    "paper_1008_2849_gb300/csrc/rs_internal.h:RS_TILE_SHAPES")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "onesweep_pairs_2^28_traffic.txt")
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal; the roofline's peak is the measured copy rate


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(rank: int) -> int:
    """Key seed of rank `rank`'s array: every replica sorts its own input."""
    return KEY_SEED + 1000 * rank


def max_over_ranks(x: float, world: int, device) -> float:
    """The maximum of `x` over all ranks (the slowest replica sets the job's
    time); `x` itself on a single rank, where no process group exists."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, n: int, seconds: float) -> float:
    """Items per second for the whole job: all ranks' items over the time."""
    return world * steps * n / seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def source_hash(paths) -> str:
    """Hash of the code in `paths`: line comments, trailing blanks and blank
    lines are left out, so that editing a comment keeps the hash.  A path
    written "file:MACRO" stands for the definition of that macro only (its
    #define line and the continuation lines after it)."""
    h = hashlib.sha256()
    for p in paths:
        path, _, macro = p.partition(":")
        with open(os.path.join(ROOT, path), encoding="utf-8") as f:
            lines = f.read().splitlines()
        if macro:
            start = next(i for i, ln in enumerate(lines) if ln.startswith("#define " + macro))
            end = start
            while lines[end].rstrip().endswith("\\"):
                end += 1
            lines = lines[start:end + 1]
        for line in lines:
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes of the scatter kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    try:
        vals = {}
        for line in open(TRAFFIC_FILE):
            line = line.split("#", 1)[0].strip()
            if "=" in line:
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
        if vals.get("source_hash") != source_hash(ONESWEEP_SOURCES):
            return None
        return float(vals["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def link_bandwidths(host_buf, dev, reps: int = 3):
    """Host->device and device->host GB/s of plain copies of `host_buf`
    (pinned) on this rank's GPU, the best of `reps` timed copies each, and
    the seconds that one copy each way takes when both run at once."""
    import torch
    d = torch.empty_like(host_buf, device=dev)
    d2 = torch.empty_like(d)
    back = torch.empty_like(host_buf).pin_memory()
    nbytes = host_buf.numel() * host_buf.element_size()
    out = []
    for dst, src in ((d, host_buf), (back, d)):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize(dev)
            best = min(best, time.perf_counter() - t0)
        out.append(nbytes / best / 1e9)
    s_up, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    duplex = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(s_up):
            d.copy_(host_buf, non_blocking=True)
        with torch.cuda.stream(s_down):
            back.copy_(d2, non_blocking=True)
        torch.cuda.synchronize(dev)
        duplex = min(duplex, time.perf_counter() - t0)
    return out[0], out[1], duplex


def host_cpu_model() -> str:
    """The host CPU's model as /proc/cpuinfo names it (best effort)."""
    try:
        fields = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                key, val = line.split(":", 1)
                fields.setdefault(key.strip(), val.strip())
        if "model name" in fields:
            return fields["model name"]
        return "implementer %s part %s" % (fields.get("CPU implementer", "?"),
                                           fields.get("CPU part", "?"))
    except OSError:
        return "unknown"


def cpu_oracle_rate(seconds_budget: float = 12.0, n_sample: int = N_PAIRS):
    """Time the CPU oracle (threaded, all host cores) on the workload itself,
    2^28 uniform pairs (seed 2), value = index: as many sorts as fit the
    time budget, at most three."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    k = inputs.keys("uniform", n_sample, seed=KEY_SEED)
    v = inputs.index_values(n_sample)
    rates = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.sort_pairs_threaded(k, v, threads)
        dt = time.perf_counter() - t0
        rates.append(n_sample / dt)
        if time.perf_counter() - t_start > seconds_budget or len(rates) >= 3:
            break
    # The plain single-threaded oracle on a smaller bounded sample, for scale.
    n_one = 1 << 23
    t0 = time.perf_counter()
    oracle.sort_pairs(k[:n_one], v[:n_one])
    single = n_one / (time.perf_counter() - t0)
    return {"value": statistics.median(rates), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d sorts of the whole workload (2^%d uniform uint32 pairs, value = "
                      "index), threaded LSD counting-sort oracle, median"
                      % (len(rates), n_sample.bit_length() - 1),
            "single_thread_value": single,
            "single_thread_sample": "one sort of 2^23 of the same pairs, plain oracle, 1 thread",
            "cpu": host_cpu_model()}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    n_sample = 1 << args.reference_sample_log2
    k = inputs.keys("uniform", n_sample, seed=KEY_SEED)
    v = inputs.index_values(n_sample)
    for _ in range(args.warmup):
        oracle.sort_pairs_threaded(k, v, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort_pairs_threaded(k, v, threads)
    dt = time.perf_counter() - t0
    value = args.steps * n_sample / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_PAIRS, "key_dist": "uniform", "seed": KEY_SEED,
                   "values": "index", "reference_sample_n": n_sample,
                   "same_config": n_sample == N_PAIRS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "each step sorts 2^%d of the workload's pairs on the host "
                                   "(threaded LSD counting-sort oracle)" % args.reference_sample_log2,
                         "cpu": host_cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_partition(args, world, rank, local):
    """One array of world * 2^28 pairs, rank r holding shard r (uniform keys,
    seed per rank, value = global index), sorted across the ranks by Alg. 2's
    partition (partition.py): local MSD pass, gather of bucket sizes,
    exchange of the items by MSD range, local sort.  A step sorts the whole
    array; value = all ranks' pairs per second over the max-over-ranks time."""
    import torch
    import torch.distributed as dist

    from paper_1008_2849_gb300 import build, clocks, partition, rs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build_library()
    rs.lib()
    n = N_PAIRS
    k_host = inputs.keys("uniform", n, seed=replica_seed(rank))
    v_host = (np.arange(n, dtype=np.uint64) + np.uint64(rank) * np.uint64(n)).astype(np.uint32)
    k_src = torch.from_numpy(k_host.view(np.int32)).to(dev)
    v_src = torch.from_numpy(v_host.view(np.int32)).to(dev)
    ops = partition.GpuOps(dev)
    total = args.warmup + args.steps
    bufs = [(k_src.clone(), v_src.clone()) for _ in range(total)]
    stream = torch.cuda.current_stream()
    for i in range(args.warmup):
        partition.partition_sort_pairs(bufs[i][0], bufs[i][1], ops)
    rs.check_stream(stream)
    received = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = rs.launch_count()
    rs.profile_enable(True)
    with clocks.ClockSampler(local) as sampler:
        ev0.record(stream)
        for i in range(args.warmup, total):
            rk, _, bounds = partition.partition_sort_pairs(bufs[i][0], bufs[i][1], ops)
            received.append(rk.numel())
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per_kind = rs.profile_read()
    rs.profile_enable(False)
    launches = rs.launch_count() - launches0
    rs.check_stream(stream)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    value = job_throughput(world, args.steps, n, elapsed_ms / 1e3)
    # Scatter-pass roofline: every step runs one MSD pass over the shard and
    # four passes over what the rank received.
    peaks, peak_src = measured_peaks()
    os_launches, os_ms = per_kind.get("onesweep", (0, 0.0))
    items = args.steps * n + 4 * sum(received)
    achieved = roofline.scatter_bytes_per_item(True) * items / (os_ms / 1e3) / 1e9 if os_ms else None
    del bufs
    torch.cuda.empty_cache()
    # End to end: the shard uploaded from pinned host memory, sorted across
    # the ranks, and this rank's part downloaded, every step.
    kin = torch.from_numpy(k_host.view(np.int32)).pin_memory()
    vin = torch.from_numpy(v_host.view(np.int32)).pin_memory()
    e2e = None
    if not args.no_e2e:
        steps_e2e = max(3, min(args.steps, 5))
        outs = []
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            kd, vd = kin.to(dev, non_blocking=True), vin.to(dev, non_blocking=True)
            rk, rv, _ = partition.partition_sort_pairs(kd, vd, ops)
            outs = (rk.cpu(), rv.cpu())
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_throughput(world, steps_e2e, n, dt), "unit": UNIT,
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * int(outs[0].numel()),
               "api": "partition.partition_sort_pairs (pinned host shard in, this rank's part out)",
               "steps": steps_e2e}
    if rank == 0:
        cs = sampler.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "sort_pairs_u32_%dx2^28_uniform_sharded" % world,
                       "n": world * n, "shard": n, "key_dist": "uniform", "values": "global index",
                       "passes": "1 MSD + 4 local", "digit_bits": 8,
                       "l2": "inputs larger than L2: every step sorts its own fresh copy",
                       "parallelism": "msd-partition (Alg. 2) over %d rank(s)" % world,
                       "bucket_ranges": [int(x) for x in bounds]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s",
                         "frac": achieved / float(peaks["hbm_gbs"]) if achieved else None,
                         "traffic": None, "kernel": "k_onesweep (all scatter passes of a step)",
                         "peak_source": peak_src + " (hbm_gbs, copy)"},
            "e2e": e2e, "cpu_baseline": None, "gpu_launches": launches,
            "clocks": {"sm_mhz": cs["sm_mhz"], "sm_max_mhz": cs["sm_max_mhz"],
                       "reasons": cs["reasons"], "samples": cs["samples"], "source": cs["source"]},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the latency, batch and serving legs (run on one GPU only)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream in the serving leg")
    ap.add_argument("--mode", choices=("auto", "sort", "partition"), default="auto",
                    help="sort: every rank sorts its own array (replicas); partition: the ranks "
                         "sort one array held in shards (Alg. 2); auto: sort on one GPU, "
                         "partition on several")
    ap.add_argument("--reference-sample-log2", type=int, default=28,
                    help="--impl reference: log2 of the pairs each step sorts on the host")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3  # at least three untimed warm-up steps

    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    mode = args.mode if args.mode != "auto" else ("partition" if world > 1 else "sort")
    if mode == "partition":
        return run_partition(args, world, rank, local)

    import torch
    import torch.distributed as dist

    from paper_1008_2849_gb300 import build, clocks, rs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build_library()
    rs.lib()

    n = N_PAIRS
    seed = replica_seed(rank)
    k_host = inputs.keys("uniform", n, seed=seed)
    v_host = inputs.index_values(n)
    dev = torch.device("cuda", local)
    k_src = torch.from_numpy(k_host.view(np.int32)).to(dev)
    v_src = torch.from_numpy(v_host.view(np.int32)).to(dev)

    total = args.warmup + args.steps
    bufs = []
    for _ in range(total):
        kb = torch.empty_like(k_src)
        vb = torch.empty_like(v_src)
        kb.copy_(k_src)
        vb.copy_(v_src)
        bufs.append((kb, vb))
    ws = rs.alloc_workspace(n, True, device=dev)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    for i in range(args.warmup):
        rs.sort_pairs_ex(bufs[i][0], bufs[i][1], ws, stream=stream)
    rs.check_stream(stream)

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = rs.launch_count()
    rs.profile_enable(True)
    with clocks.ClockSampler(local) as sampler:
        ev0.record(stream)
        for i in range(args.warmup, total):
            rs.sort_pairs_ex(bufs[i][0], bufs[i][1], ws, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per_kind = rs.profile_read()
    rs.profile_enable(False)
    launches = rs.launch_count() - launches0
    rs.check_stream(stream)
    elapsed_ms = ev0.elapsed_time(ev1)

    elapsed_ms = max_over_ranks(elapsed_ms, world, dev)
    value = job_throughput(world, args.steps, n, elapsed_ms / 1e3)

    # Roofline of the dominant kernel: the scatter pass.
    peaks, peak_src = measured_peaks()
    os_launches, os_ms = per_kind.get("onesweep", (0, 0.0))
    hist_launches, hist_ms = per_kind.get("hist4", (0, 0.0))
    algo_bytes = roofline.scatter_bytes_per_item(True) * n   # per scatter launch
    achieved = algo_bytes / (os_ms / os_launches / 1e3) / 1e9 if os_launches else None
    peak = float(peaks["hbm_gbs"])
    traffic = recorded_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "kernel": "k_onesweep (pairs, default tile shape)", "peak_source": peak_src + " (hbm_gbs, copy)",
            "nominal_peak": NOMINAL_HBM_GBS,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS if achieved else None,
            "avg_launch_ms": os_ms / os_launches if os_launches else None,
            "algorithmic_bytes_per_launch": algo_bytes,
            "hist_avg_launch_ms": hist_ms / hist_launches if hist_launches else None,
            "hist_achieved_gbs": (roofline.histogram_bytes_per_item() * n / (hist_ms / hist_launches / 1e3) / 1e9)
            if hist_launches else None,
            "whole_sort_gbs": roofline.sort_bytes_per_item(True) * n * args.steps / (elapsed_ms / 1e3) / 1e9,
            "per_kind_ms": {k: v[1] / max(v[0], 1) for k, v in per_kind.items() if v[0]}}

    # Release the step buffers before the end-to-end and CPU legs.
    del bufs
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        # Host arrays in pinned memory; every step uploads its input, sorts it
        # and downloads its result.  One rs_sort_pairs_host_batch call runs
        # all steps with rotating device buffer sets, so that step i+1's upload
        # and step i-1's download overlap step i's sort.
        kin = torch.from_numpy(k_host.view(np.int32)).pin_memory()
        vin = torch.from_numpy(v_host.view(np.int32)).pin_memory()
        outs = [(torch.empty_like(kin).pin_memory(), torch.empty_like(vin).pin_memory())
                for _ in range(2)]

        def host_batch(steps):
            rs.sort_pairs_host_batch([kin] * steps, [vin] * steps,
                                     [outs[i % 2][0] for i in range(steps)],
                                     [outs[i % 2][1] for i in range(steps)])
        host_batch(2)
        e2e_steps = max(3, min(args.steps, 10))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        host_batch(e2e_steps)
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_throughput(world, e2e_steps, n, dt), "unit": UNIT,
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
               "api": "rs_sort_pairs_host_batch (pinned host buffers, all steps in one call)",
               "steps": e2e_steps}
        # For comparison: one synchronous rs_sort_pairs_host call per array.
        rs.sort_pairs_host(kin, vin, outs[0][0], outs[0][1])
        serial_steps = 3
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(serial_steps):
            rs.sort_pairs_host(kin, vin, outs[0][0], outs[0][1])
        dt1 = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e["one_call_per_array"] = {"value": job_throughput(world, serial_steps, n, dt1),
                                     "api": "rs_sort_pairs_host"}
        # The host link bounds these numbers: time the same bytes through
        # plain pinned copies.  One array at a time, copies and the
        # device-timed sort run in series; pipelined, a step needs at least
        # the longer of the sort and one upload with one download at once.
        del outs
        h2d, d2h, duplex_half = link_bandwidths(kin, dev)
        sort_s = elapsed_ms / 1e3 / args.steps
        serial_s = 8 * n / (h2d * 1e9) + 8 * n / (d2h * 1e9) + sort_s
        pipe_s = max(2 * duplex_half, sort_s)  # keys and values: two copies each way
        e2e.update({"link_h2d_gbs": h2d, "link_d2h_gbs": d2h,
                    "link_gbs_each_way_at_once": 4 * n / duplex_half / 1e9,
                    "serial_bound": n / serial_s, "pipelined_bound": n / pipe_s,
                    "frac_of_pipelined_bound": (e2e["value"] / world) / (n / pipe_s)})

    # The metric's other parts, on one GPU: the 2^20-key latency (config 1),
    # the batched sort (config 4 rescaled to 2^28 pairs) and the serving
    # loop's p50/p99 (a seeded prefix of the config-5 stream).
    extras = {}
    if world == 1 and not args.no_extras:
        from paper_1008_2849_gb300 import bench_extras
        torch.cuda.empty_cache()
        extras["latency_2^20_keys"] = bench_extras.latency_keys_2pow20(local)
        torch.cuda.empty_cache()
        extras["batch"] = bench_extras.batch_2pow28(local)
        torch.cuda.empty_cache()
        extras["serve"] = bench_extras.serve_stream(local, requests=args.serve_requests)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate()

    if rank == 0:
        cs = sampler.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "key_dist": "uniform", "seed": KEY_SEED,
                       "values": "index", "passes": 4, "digit_bits": 8,
                       "l2": "inputs larger than L2: every step sorts its own fresh 2 GiB copy",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": launches,
            "latency_2^20_keys_ms": (extras["latency_2^20_keys"]["call_ms"]
                                     if "latency_2^20_keys" in extras else None),
            **extras,
            "clocks": {"sm_mhz": cs["sm_mhz"], "sm_max_mhz": cs["sm_max_mhz"],
                       "reasons": cs["reasons"], "samples": cs["samples"], "source": cs["source"]},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
