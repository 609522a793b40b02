"""The metric's other two parts, measured inside bench.py's run on one GPU:
the latency of the small keys-only sort, the batched segmented sort against
a loop of per-array sorts, and p50/p99 latency of the serving loop against
serial plain sorts.  Each leg samples the SM clocks while it runs.

* latency: 2^20 uniform uint32 keys (seed 1), keys only, four 8-bit LSD
  passes; device time (CUDA events) of one rs_sort_keys_ex and of one replay
  of a captured graph of it, median over the steps.  The 4 MiB array stays
  in the 129 MB L2 between steps, so this is a latency, not a roofline case.
* batch: 4096 arrays of (uint32 key, uint32 value = index inside the array),
  sizes log-uniform on [2^8, 2^22] (seed 10), rescaled to 2^28 pairs in
  total, uniform keys; one graph launch of rs_sort_pairs_segmented_ex per
  step, against one rs_sort_pairs_ex call per array on one stream.  Every
  step sorts a fresh copy (restored outside the timed events).
* serve: the first `requests` requests of the serving stream (70 % keys
  only, 30 % key-value, sizes floor(10^U) with U uniform on [3, 8], uniform
  or AND-of-2 keys, seed 11) with Poisson arrivals at 0.8 times the measured
  capacity of serial plain sorts, served in real time under a 60 GB budget by
  the continuous-batching server and by serial plain sorts.
"""
from __future__ import annotations

import statistics

import numpy as np


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _clocks(sampler) -> dict:
    cs = sampler.summary()
    return {"sm_mhz": cs["sm_mhz"], "sm_max_mhz": cs["sm_max_mhz"], "reasons": cs["reasons"],
            "samples": cs["samples"]}


def latency_keys_2pow20(device_index: int, steps: int = 20, warmup: int = 5) -> dict:
    import torch

    from paper_1008_2849_gb300 import clocks, inputs, rs
    n = 1 << 20
    src = torch.from_numpy(inputs.keys("uniform", n, seed=1).view(np.int32)).cuda()
    k = torch.empty_like(src)
    ws = rs.alloc_workspace(n, False)
    stream = torch.cuda.current_stream()
    graph = rs.Graph(k, None, None, ws)

    def timed(fn):
        out = []
        for i in range(warmup + steps):
            k.copy_(src)
            e0, e1 = _events(torch)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= warmup:
                out.append(e0.elapsed_time(e1))
        rs.check_stream(stream)
        return statistics.median(out)

    with clocks.ClockSampler(device_index) as sampler:
        call_ms = timed(lambda: rs.sort_keys_ex(k, ws, stream=stream))
        graph_ms = timed(lambda: graph.launch(stream))
    graph.close()
    ok = bool(torch.equal(k.cpu(), torch.from_numpy(
        np.sort(src.cpu().numpy().view(np.uint32)).view(np.int32))))
    return {"call_ms": call_ms, "graph_replay_ms": graph_ms, "keys": n, "steps": steps,
            "workload": "2^20 uniform uint32 keys, seed 1, keys only, 4 x 8-bit passes "
                        "(L2-resident between steps)",
            "sorted": ok, "clocks": _clocks(sampler)}


def batch_2pow28(device_index: int, steps: int = 5, warmup: int = 3, loop_steps: int = 2) -> dict:
    import torch

    from paper_1008_2849_gb300 import clocks, inputs, rs
    k_np, v_np, off_np = inputs.segmented_batch(4096, 8, 22, seed=10, scale_to=1 << 28)
    n = int(k_np.size)
    k = torch.from_numpy(k_np.view(np.int32)).cuda()
    v = torch.from_numpy(v_np.view(np.int32)).cuda()
    off = torch.from_numpy(off_np.view(np.int32)).cuda()
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    stream = torch.cuda.current_stream()

    def arm(fn, nsteps):
        out = []
        for i in range(warmup + nsteps):
            kb.copy_(k)
            vb.copy_(v)
            e0, e1 = _events(torch)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= warmup:
                out.append(e0.elapsed_time(e1))
        rs.check_stream(stream)
        return float(np.mean(out))

    graph = rs.Graph(kb, vb, off)
    offs = off_np.astype(np.int64)
    ws = rs.alloc_workspace(int(np.diff(offs).max()), True)
    views = [(kb[offs[s]:offs[s + 1]], vb[offs[s]:offs[s + 1]]) for s in range(4096)
             if offs[s + 1] > offs[s]]

    def loop():
        for kk, vv in views:
            rs.sort_pairs_ex(kk, vv, ws, stream=stream)

    with clocks.ClockSampler(device_index) as sampler:
        l0 = rs.launch_count()
        batch_ms = arm(lambda: graph.launch(stream), steps)
        kernels = (rs.launch_count() - l0) // (warmup + steps)
        loop_ms = arm(loop, loop_steps)
    graph.close()
    return {"value": n / (batch_ms / 1e3), "unit": "pairs/s", "ms_per_step": batch_ms,
            "kernels_per_step": int(kernels), "api": "rs_graph_launch (rs_sort_pairs_segmented_ex)",
            "loop": {"value": n / (loop_ms / 1e3), "ms_per_step": loop_ms,
                     "api": "rs_sort_pairs_ex per array, one stream", "steps": loop_steps},
            "batched_over_loop": loop_ms / batch_ms, "n_pairs": n, "segments": 4096,
            "steps": steps,
            "workload": "4096 arrays, sizes log-uniform [2^8, 2^22] (seed 10), rescaled to "
                        "2^28 pairs, uniform keys, value = index in the array",
            "clocks": _clocks(sampler)}


def serve_stream(device_index: int, requests: int = 2000, load: float = 0.8,
                 calibrate: int = 200, budget_gb: float = 60.0) -> dict:
    from paper_1008_2849_gb300 import clocks, serve
    ex = serve.GpuExecutor(streams=4, device=device_index)
    budget = int(budget_gb * 1e9)
    warm = [serve.Request(10**9 + i, m, wv, "uniform", i) for i, (m, wv) in
            enumerate([(1000, False), (1000, True), (10**6, False), (10**6, True)])]
    serve.SortServer(ex, budget_bytes=budget).run(warm, realtime=False)
    base = serve.make_requests(requests, 11)
    with clocks.ClockSampler(device_index) as sampler:
        cal = serve.SerialServer(ex).run(base[:calibrate], realtime=False)
        mean_n = sum(r.n for r in base) / len(base)
        rate = load * cal["items_per_s"] / mean_n
        reqs = serve.make_requests(requests, 11, rate_per_s=rate)
        live = serve.SortServer(ex, budget_bytes=budget, max_inflight=8).run(reqs, realtime=True)
        serial = serve.SerialServer(ex).run(reqs, realtime=True)
    ms = 1e3
    return {"p50_ms": live["p50_s"] * ms, "p99_ms": live["p99_s"] * ms,
            "items_per_s": live["items_per_s"], "launches": live["launches"],
            "peak_bytes": live["peak_bytes"], "budget_bytes": budget,
            "serial": {"p50_ms": serial["p50_s"] * ms, "p99_ms": serial["p99_s"] * ms,
                       "items_per_s": serial["items_per_s"]},
            "p99_serial_over_server": serial["p99_s"] / live["p99_s"],
            "offered_load": load, "arrival_rate_per_s": rate,
            "serial_capacity_items_per_s": cal["items_per_s"], "requests": requests,
            "workload": "first %d requests of the serving stream (seed 11): 70%% keys / 30%% "
                        "pairs (uint32), sizes floor(10^U), U~U[3,8], uniform or AND-2 keys, "
                        "Poisson arrivals in real time" % requests,
            "clocks": _clocks(sampler)}
