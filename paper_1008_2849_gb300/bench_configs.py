"""Benchmarks of the keys-only latency case and of the distribution sweep.

    python -m paper_1008_2849_gb300.bench_configs [--steps K] [--warmup W]

1. Keys only, 2^20 uniform uint32 keys (seed 1), four 8-bit LSD passes:
   device time of one rs_sort_keys_ex (median of K), so a latency.  The array
   is 4 MiB and stays in L2 between steps: this case is not an HBM roofline
   case.  The same input is also timed in the MSD-first order of Alg. 2, and
   uniform pairs of 2^14..2^21 items in both orders; each also as the replay
   of a captured graph (rs_graph_launch), which removes the host's launch
   overhead from the device timeline.
2. Distribution sweep at 2^27 pairs (value = index; seeds 3, 4, ...):
   uniform; AND of 2, 3 and 4 uniform words; 256 distinct values; all keys
   equal; sorted; reverse sorted; low 16 bits only.  Each step sorts a fresh
   copy (1 GiB, larger than L2) with rs_sort_pairs_ex; reported are pairs/s
   (median step) and the number of scatter passes that ran -- a digit that is
   the same for every key makes its pass the identity, and it is skipped.
3. Typed keys at 2^27 pairs of random 32-bit words (seed 21), read as
   signed integers and as IEEE floats (rs_sort_typed_ex); and float-key
   pairs of 2^14..2^26 items with two scatter-pass instances per pass
   against one (RS_TUNE_TYPED_SPLIT), as graph replays.
4. 64-bit keys with 32-bit values, 2^27 pairs of random words (seed 22),
   eight passes (rs_sort64_ex).
5. Wide items through rs_sort_kv_ex at 2^27 items of random words (seed
   23): 32-bit keys with 64-bit values (four passes), 64-bit keys (unsigned
   and IEEE binary64) with 64-bit values and signed 64-bit keys alone (eight
   passes).
6. Digit width of the whole-array sort: four 8-bit passes (rs_sort_pairs_ex,
   rs_sort_keys_ex) against three 11/11/10-bit passes (rs_sort_digits11_ex)
   with every tile shape of its scatter kernel, pairs and keys only of
   2^20..2^28 uniform keys (seed 25), each step on a fresh copy; with the
   device time of each of its kernels (rs_profile_*) for the default shape.

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys

import numpy as np

DISTS = ("uniform", "and2", "and3", "and4", "distinct256", "equal", "sorted", "reverse", "low16")


def _timed(torch, stream, fn, restore, steps, warmup):
    times = []
    for i in range(warmup + steps):
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args(argv)

    import torch

    from paper_1008_2849_gb300 import build, inputs, rs
    build.build_library()
    rs.lib()
    stream = torch.cuda.current_stream()
    out = {"metric": "sort throughput and latency per configuration", "unit": "pairs/s"}

    # 1. keys only, 2^20: the four LSD passes (as the configuration states),
    # and the MSD-first order of Alg. 2 on the same input (same result).
    n = 1 << 20
    k = torch.from_numpy(inputs.keys("uniform", n, seed=1).view(np.int32)).cuda()
    kb = torch.empty_like(k)
    ws = rs.alloc_workspace(n, False)
    cls = rs.size_class(n)
    old_msd = rs.tune_get_class(cls, "msd")
    for msd, name in ((0, "keys_2^20_uniform_seed1"), (1, "keys_2^20_uniform_seed1_msd_first")):
        rs.tune_set_class(cls, "msd", msd)
        ms = _timed(torch, stream, lambda: rs.sort_keys_ex(kb, ws, stream), lambda: kb.copy_(k),
                    a.steps, a.warmup)
        g = rs.Graph(kb, None, None, ws)
        ms_graph = _timed(torch, stream, lambda: g.launch(stream), lambda: kb.copy_(k), a.steps,
                          a.warmup)
        g.close()
        rs.check_stream()
        out[name] = {"ms": ms, "keys_per_s": n / (ms / 1e3), "graph_replay_ms": ms_graph}
    rs.tune_set_class(cls, "msd", old_msd)
    del k, kb, ws

    # Mid-size pairs: LSD passes vs MSD-first order.
    mid = {}
    for lg in (14, 16, 18, 20, 21):
        n = 1 << lg
        k = torch.from_numpy(inputs.keys("uniform", n, seed=40 + lg).view(np.int32)).cuda()
        v = torch.arange(n, dtype=torch.int32, device="cuda")
        kb, vb = torch.empty_like(k), torch.empty_like(v)
        ws = rs.alloc_workspace(n, True)
        cls = rs.size_class(n)
        old_msd = rs.tune_get_class(cls, "msd")
        row = {}
        for msd in (0, 1):
            rs.tune_set_class(cls, "msd", msd)

            def restore():
                kb.copy_(k)
                vb.copy_(v)
            ms = _timed(torch, stream, lambda: rs.sort_pairs_ex(kb, vb, ws, stream), restore,
                        a.steps, a.warmup)
            g = rs.Graph(kb, vb, None, ws)
            ms_graph = _timed(torch, stream, lambda: g.launch(stream), restore, a.steps, a.warmup)
            g.close()
            rs.check_stream()
            row["msd_first" if msd else "lsd"] = {"ms": ms, "pairs_per_s": n / (ms / 1e3),
                                                  "graph_replay_ms": ms_graph}
        rs.tune_set_class(cls, "msd", old_msd)
        mid["2^%d" % lg] = row
        del k, v, kb, vb, ws
    out["pairs_mid_sizes_lsd_vs_msd_first"] = mid

    # Keys only at 2^27 (uniform, seed 3): 8 B per key per pass.
    n = 1 << 27
    k = torch.from_numpy(inputs.keys("uniform", n, seed=3).view(np.int32)).cuda()
    kb = torch.empty_like(k)
    ws = rs.alloc_workspace(n, False)
    ms = _timed(torch, stream, lambda: rs.sort_keys_ex(kb, ws, stream), lambda: kb.copy_(k),
                a.steps, a.warmup)
    rs.check_stream()
    out["keys_2^27_uniform"] = {"ms": ms, "keys_per_s": n / (ms / 1e3)}
    del k, kb, ws

    # 2. distribution sweep, 2^27 pairs
    n = 1 << 27
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    kb, vb = torch.empty_like(v), torch.empty_like(v)
    ws = rs.alloc_workspace(n, True)
    sweep = {}
    for i, dist in enumerate(DISTS):
        k = torch.from_numpy(inputs.keys(dist, n, seed=3 + i).view(np.int32)).cuda()

        def restore():
            kb.copy_(k)
            vb.copy_(v)
        rs.profile_enable(True)
        rs.profile_read()
        ms = _timed(torch, stream, lambda: rs.sort_pairs_ex(kb, vb, ws, stream), restore,
                    a.steps, a.warmup)
        launches, _ = rs.profile_read().get("onesweep", (0, 0.0))
        rs.profile_enable(False)
        rs.check_stream()
        # Scatter-pass launches per sort; a launch whose pass is skipped
        # returns at once (it is still counted as a launch).
        hist = rs.digit_histograms(k).cpu().numpy().view(np.uint32)
        sweep[dist] = {"seed": 3 + i, "ms": ms, "pairs_per_s": n / (ms / 1e3),
                       "passes_executed": _executed_passes(hist, n),
                       "scatter_launches_per_sort": launches // (a.steps + a.warmup)}
        del k
    out["pairs_2^27_distributions"] = sweep

    # 3. typed keys (signed integers, IEEE floats), 2^27 pairs of random words
    typed = {}
    for key_type in ("i32", "f32"):
        k = torch.from_numpy(inputs.keys("uniform", n, seed=21).view(np.int32)).cuda()

        def restore():
            kb.copy_(k)
            vb.copy_(v)
        ms = _timed(torch, stream, lambda: rs.sort_typed_ex(kb, vb, key_type, ws, stream), restore,
                    a.steps, a.warmup)
        rs.check_stream()
        typed[key_type] = {"ms": ms, "pairs_per_s": n / (ms / 1e3)}
        del k
    out["pairs_2^27_typed_keys"] = typed
    del kb, vb, ws

    # 3b. typed keys across sizes: two scatter-pass instances per pass (the
    # middle passes without the key map) against one mapping instance per
    # pass (half the launches), each as the replay of a captured graph.
    out["typed_f32_pairs_split_vs_single"] = _typed_split_sweep(torch, rs, inputs, stream, a)

    # 4. 64-bit keys (eight passes) with 32-bit values, 2^27 pairs of random
    # words (seed 22): 1 GiB of keys.
    hi = inputs.splitmix32(22, n, 0).astype(np.uint64)
    lo = inputs.splitmix32(22, n, 1).astype(np.uint64)
    k = torch.from_numpy(((hi << np.uint64(32)) | lo).view(np.int64)).cuda()
    del hi, lo
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    nbytes = rs.workspace_bytes64(n, True)
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ws = raw[(-raw.data_ptr()) % 256:][:nbytes]

    def restore():
        kb.copy_(k)
        vb.copy_(v)
    ms = _timed(torch, stream, lambda: rs.sort64_ex(kb, vb, ws, stream), restore, a.steps,
                a.warmup)
    rs.check_stream()
    out["pairs_2^27_key64_value32"] = {"ms": ms, "pairs_per_s": n / (ms / 1e3),
                                       "bytes_per_pair_per_pass": 24, "passes": 8}
    del kb, vb, ws, raw

    # 5. wide items (rs_sort_kv_ex), 2^27 items of random words (seed 23)
    i64 = torch.arange(n, dtype=torch.int64, device="cuda")
    wide = {}
    for key_type, value_bits in (("u32", 64), ("u64", 64), ("f64", 64), ("i64", 0)):
        kw = 8 if key_type.endswith("64") else 4
        lo = inputs.splitmix32(23, n, 0)
        if kw == 8:
            hi = inputs.splitmix32(23, n, 1).astype(np.uint64)
            k = torch.from_numpy(((hi << np.uint64(32)) | lo.astype(np.uint64)).view(np.int64))
            del hi
        else:
            k = torch.from_numpy(lo.view(np.int32))
        k = k.cuda()
        del lo
        vw = i64 if value_bits == 64 else None
        kb = torch.empty_like(k)
        vb = None if vw is None else torch.empty_like(vw)
        nbytes = rs.workspace_bytes_kv(n, key_type, value_bits)
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ws = raw[(-raw.data_ptr()) % 256:][:nbytes]

        def restore():
            kb.copy_(k)
            if vb is not None:
                vb.copy_(vw)
        ms = _timed(torch, stream, lambda: rs.sort_kv_ex(kb, vb, key_type, ws, stream), restore,
                    a.steps, a.warmup)
        rs.check_stream()
        passes = 8 if kw == 8 else 4
        per_pass = 2 * (kw + value_bits // 8)
        wide["%s_keys_%d_bit_values" % (key_type, value_bits)] = {
            "ms": ms, "items_per_s": n / (ms / 1e3), "passes": passes,
            "bytes_per_item_per_pass": per_pass,
            "scatter_tb_per_s": n * per_pass * passes / (ms / 1e3) / 1e12}
        del k, kb, vb, ws, raw
    out["items_2^27_wide"] = wide
    del i64

    # 6. four 8-bit passes against three 11/11/10-bit ones.
    out["digits11_vs_8"] = _digits_sweep(torch, rs, inputs, stream, a)
    print(json.dumps(out), flush=True)
    return 0


def _digits_sweep(torch, rs, inputs, stream, a):
    rows = {}
    old = rs.tune_get("d11_shape")
    try:
        for lg in (20, 22, 24, 26, 28):
            n = 1 << lg
            k = inputs.keys_torch("uniform", n, seed=25)
            v = torch.arange(n, dtype=torch.int32, device="cuda")
            kb, vb = torch.empty_like(k), torch.empty_like(v)

            def restore():
                kb.copy_(k)
                vb.copy_(v)
            for pairs in (True, False):
                row = {}
                ws = rs.alloc_workspace(n, pairs)
                if pairs:
                    fn8 = lambda: rs.sort_pairs_ex(kb, vb, ws, stream)  # noqa: E731
                else:
                    fn8 = lambda: rs.sort_keys_ex(kb, ws, stream)  # noqa: E731
                row["digits8_ms"] = _timed(torch, stream, fn8, restore, a.steps, a.warmup)
                del ws
                ws = rs.alloc_workspace_digits11(n, pairs)
                vv = vb if pairs else None
                for shape in range(4):
                    rs.tune_set("d11_shape", shape)
                    row["digits11_shape%d_ms" % shape] = _timed(
                        torch, stream, lambda: rs.sort_digits11_ex(kb, vv, ws, stream), restore,
                        a.steps, a.warmup)
                rs.tune_set("d11_shape", old)
                restore()
                rs.profile_enable(True)
                rs.profile_read()
                rs.sort_digits11_ex(kb, vv, ws, stream)
                torch.cuda.synchronize()
                prof = rs.profile_read()
                rs.profile_enable(False)
                row["digits11_kernels_ms"] = {kind: ms for kind, (cnt, ms) in prof.items() if cnt}
                rs.check_stream()
                rows["%s_2^%d" % ("pairs" if pairs else "keys", lg)] = row
                del ws
            del k, v, kb, vb
            torch.cuda.empty_cache()
    finally:
        rs.tune_set("d11_shape", old)
    return rows


def _typed_split_sweep(torch, rs, inputs, stream, a):
    rows = {}
    old = rs.tune_get("typed_split")
    try:
        for lg in (14, 16, 18, 20, 22, 24, 26):
            n = 1 << lg
            k = torch.from_numpy(inputs.keys("uniform", n, seed=24 + lg).view(np.int32)).cuda()
            v = torch.arange(n, dtype=torch.int32, device="cuda")
            kb, vb = torch.empty_like(k), torch.empty_like(v)
            ws = rs.alloc_workspace(n, True)
            row = {}
            for name, split_min in (("two_instances", 0), ("one_instance", 0x7FFFFFFF)):
                rs.tune_set("typed_split", split_min)
                rs.sort_typed_ex(kb, vb, "f32", ws, stream)  # first use outside capture
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                side = torch.cuda.Stream()
                with torch.cuda.graph(g, stream=side):
                    rs.sort_typed_ex(kb, vb, "f32", ws, side)

                def restore():
                    kb.copy_(k)
                    vb.copy_(v)
                row[name + "_ms"] = _timed(torch, stream, g.replay, restore, a.steps, a.warmup)
                del g
            rs.check_stream()
            rows["2^%d" % lg] = row
            del k, v, kb, vb, ws
    finally:
        rs.tune_set("typed_split", old)
    return rows


def _executed_passes(hist, n):
    """Scatter passes that move data, from the digit histograms: a digit whose
    histogram has one bucket holding all n keys is the identity and skipped;
    one identity pass is added back when needed to keep the count even (the
    result must end in the caller's buffer)."""
    moving = int(sum(1 for p in range(4) if int(hist[p].max()) != n))
    return moving + (moving & 1)


if __name__ == "__main__":
    sys.exit(main())
