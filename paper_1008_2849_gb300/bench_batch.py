"""Benchmark of the batched (segmented) sort against a loop of per-array sorts.

    python -m paper_1008_2849_gb300.bench_batch [--steps K] [--warmup W] [--full]
           [--tuning tuning.json]

Workload: 4096 independent arrays of (uint32 key, uint32 value = index inside
the array), sizes log-uniform on [2^8, 2^22] (seed 10), uniform keys, offsets
as a uint32 segment table.  By default the drawn sizes are rescaled so the
batch totals about 2^28 pairs; --full keeps the drawn sizes (about 1.89e9
pairs, 15 GB of keys and values).

Arms, each timed with CUDA events over exactly K steps, every step on a fresh
copy of the batch (restored outside the timed events):
  batched   one captured graph of rs_sort_pairs_segmented_ex (one launch);
  loop      one rs_sort_pairs_ex call per array, in order, on one stream.
Prints one JSON line with both throughputs (pairs/s) and their ratio.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--full", action="store_true")
    ap.add_argument("--tuning", default=None, help="autotuner table to apply first")
    ap.add_argument("--no-loop", action="store_true", help="skip the per-array loop arm")
    a = ap.parse_args(argv)

    import torch

    from paper_1008_2849_gb300 import autotune, build, inputs, rs
    build.build_library()
    rs.lib()
    if a.tuning:
        autotune.apply(autotune.load(a.tuning))
    k_np, v_np, off_np = inputs.segmented_batch(4096, 8, 22, seed=10,
                                                scale_to=None if a.full else 1 << 28)
    n = k_np.size
    k = torch.from_numpy(k_np.view(np.int32)).cuda()
    v = torch.from_numpy(v_np.view(np.int32)).cuda()
    off = torch.from_numpy(off_np.view(np.int32)).cuda()
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    stream = torch.cuda.current_stream()

    def run_arm(step_fn):
        times = []
        for i in range(a.warmup + a.steps):
            kb.copy_(k)
            vb.copy_(v)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            step_fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= a.warmup:
                times.append(e0.elapsed_time(e1))
        rs.check_stream(stream)
        return times

    graph = rs.Graph(kb, vb, off)
    launches0 = rs.launch_count()
    t_batch = run_arm(lambda: graph.launch(stream))
    batch_launches = (rs.launch_count() - launches0) // (a.warmup + a.steps)
    # Spot-check the result of the last step against per-segment invariants.
    ku = kb.long() & 0xFFFFFFFF
    seg = torch.repeat_interleave(torch.arange(4096, device="cuda"),
                                  (off[1:].long() - off[:-1].long()))
    same = seg[1:] == seg[:-1]
    ok = bool(((ku[1:] >= ku[:-1]) | ~same).all())
    graph.close()

    line = {"metric": "32-bit key-value pairs sorted/s (batched segmented sort)",
            "unit": "pairs/s", "n_pairs": n, "segments": 4096, "steps": a.steps,
            "warmup": a.warmup, "workload": "4096 arrays, sizes log-uniform [2^8, 2^22], seed 10"
            + ("" if a.full else ", rescaled to 2^28 pairs"),
            "batched": {"value": n / (np.mean(t_batch) / 1e3), "ms_per_step": float(np.mean(t_batch)),
                        "kernels_per_step": int(batch_launches), "api": "rs_graph_launch"},
            "sorted_within_segments": ok}
    if not a.no_loop:
        offs = off_np.astype(np.int64)
        ws = rs.alloc_workspace(int(np.diff(offs).max()), True)
        views = [(kb[offs[s]:offs[s + 1]], vb[offs[s]:offs[s + 1]]) for s in range(4096)
                 if offs[s + 1] > offs[s]]

        def loop():
            for kk, vv in views:
                rs.sort_pairs_ex(kk, vv, ws, stream=stream)
        t_loop = run_arm(loop)
        line["loop"] = {"value": n / (np.mean(t_loop) / 1e3), "ms_per_step": float(np.mean(t_loop)),
                        "api": "rs_sort_pairs_ex per array"}
        line["batched_over_loop"] = line["batched"]["value"] / line["loop"]["value"]
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
