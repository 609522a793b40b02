"""Benchmark of the serving loop against serial plain sorts.

    python -m paper_1008_2849_gb300.bench_serve [--requests 20000] [--load 0.8]

Workload: a Poisson stream of sort requests, 70 % keys only and 30 % key-value
(uint32), sizes floor(10^U) with U uniform on [3, 8], uniform or AND-of-2 keys
with equal probability (seed 11), admitted under a 60 GB device-memory budget.

1. The capacity of serial plain sorts (one request at a time, each sorted
   alone and waited for) is measured on the first `--calibrate` requests,
   all present at time 0; the arrival rate is then set so that the offered
   load is `--load` times that capacity.
2. The server and the serial baseline each serve the same arrival stream in
   real time; both report p50 / p99 latency (arrival to completion) and
   items per second.
3. Both also serve all requests present at time 0 (saturated throughput).

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--calibrate", type=int, default=400)
    ap.add_argument("--budget-gb", type=float, default=60.0)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--no-saturated", action="store_true")
    a = ap.parse_args(argv)

    from paper_1008_2849_gb300 import serve

    ex = serve.GpuExecutor(streams=a.streams)
    base = serve.make_requests(a.requests, 11)
    # Warm-up: one small and one large sort of each kind (lazy loading, attributes).
    warm = [serve.Request(10**9 + i, n, wv, "uniform", i) for i, (n, wv) in
            enumerate([(1000, False), (1000, True), (10**6, False), (10**6, True)])]
    serve.SortServer(ex, budget_bytes=int(a.budget_gb * 1e9)).run(warm, realtime=False)

    cal = serve.SerialServer(ex).run(base[:a.calibrate], realtime=False)
    mean_n = sum(r.n for r in base) / len(base)
    rate = a.load * cal["items_per_s"] / mean_n  # requests per second
    reqs = serve.make_requests(a.requests, 11, rate_per_s=rate)

    srv = serve.SortServer(ex, budget_bytes=int(a.budget_gb * 1e9), max_inflight=8)
    live = srv.run(reqs, realtime=True)
    serial = serve.SerialServer(ex).run(reqs, realtime=True)
    line = {"metric": "sort requests served: p50/p99 latency and items/s",
            "workload": "%d requests, 70%% keys / 30%% pairs (uint32), sizes 10^U with U~U[3,8], "
                        "uniform or AND-2 keys, seed 11, Poisson arrivals" % a.requests,
            "offered_load": a.load, "arrival_rate_per_s": rate,
            "serial_capacity_items_per_s": cal["items_per_s"],
            "server": {k: live[k] for k in ("p50_s", "p99_s", "items_per_s", "wall_s", "launches",
                                            "peak_bytes", "budget_bytes")},
            "serial": {k: serial[k] for k in ("p50_s", "p99_s", "items_per_s", "wall_s")}}
    if not a.no_saturated:
        sat = serve.make_requests(a.requests, 11)
        s1 = serve.SortServer(ex, budget_bytes=int(a.budget_gb * 1e9), max_inflight=8).run(
            sat, realtime=False)
        s2 = serve.SerialServer(ex).run(sat, realtime=False)
        line["saturated"] = {"server_items_per_s": s1["items_per_s"],
                             "serial_items_per_s": s2["items_per_s"],
                             "server_wall_s": s1["wall_s"], "serial_wall_s": s2["wall_s"]}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
