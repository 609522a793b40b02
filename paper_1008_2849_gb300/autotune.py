"""Autotuner of the sort's launch shapes, per size class.

For every size class of the library (by item count: <= 2^13, <= 2^16, <= 2^20,
<= 2^24, <= 2^28, larger; for a segmented sort the average segment), it times
captured CUDA graphs (rs_graph_*) of a representative synthetic workload
under every candidate setting and keeps the fastest:

* whole arrays: the tile shape of the scatter passes, for key-value and for
  keys-only sorts; up to 2^21 items, the MSD-first order of Alg. 2 (one pass
  by the top digit, then on-chip bucket sorts) or the four LSD passes; from
  2^24 items, four passes of 8-bit digits or three of 11/11/10 bits; for
  arrays up to 8192 items, which take the one-CTA sort, and at which digit
  width;
* segmented batches: the tile shape of the segmented scatter passes and the
  largest segment sorted by the one-CTA sort (4096 or 8192); for batches of
  short arrays the largest segment sorted by the one-warp sort and the digit
  width of the on-chip sorts (4 bits, eight passes, or 8 bits, four passes).

Results never depend on the settings, only speed does.  The table is JSON:

    {"device": "...", "classes": {"3": {"tile_pairs": 3, "tile_keys": 3, ...}}}

    python -m paper_1008_2849_gb300.autotune --out tuning.json [--quick]
    rs_tuning = autotune.load("tuning.json"); autotune.apply(rs_tuning)
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

# Representative item counts per size class (whole arrays).
CLASS_SIZES = {1: 1 << 16, 2: 1 << 20, 3: 1 << 24, 4: 1 << 27}
MSD_MAX_ITEMS = 256 * 8192  # largest whole array the MSD-first order is tried for
DIGITS11_MIN_ITEMS = 1 << 24  # smallest whole array the 11-bit-digit order is tried for


def _time_graph(rs, torch, graph, restore, reps):
    """Median device time (ms) of `reps` graph replays, each on fresh input."""
    times = []
    stream = torch.cuda.current_stream()
    for i in range(reps + 1):
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:  # the first replay is a warm-up
            times.append(e0.elapsed_time(e1))
    rs.check_stream()
    return float(np.median(times))


def tune_whole(rs, torch, inputs, reps=3, quick=False):
    shapes = list(range(len(rs.tile_shapes())))
    out = {}
    for cls, n in CLASS_SIZES.items():
        if quick and n > (1 << 24):
            continue
        k = torch.from_numpy(inputs.keys("uniform", n, seed=200 + cls).view(np.int32)).cuda()
        v = torch.arange(n, dtype=torch.int32, device="cuda")
        kb, vb = torch.empty_like(k), torch.empty_like(v)
        best = {}
        saved = {kn: rs.tune_get_class(cls, kn)
                 for kn in ("tile_pairs", "tile_keys", "msd", "digits")}
        rs.tune_set_class(cls, "digits", 8)  # shapes are timed on the 8-bit passes
        rs.tune_set_class(cls, "msd", 0)  # shapes are timed on the four LSD passes
        for pairs in (True, False):
            knob = "tile_pairs" if pairs else "tile_keys"
            old = rs.tune_get_class(cls, knob)
            res = {}
            for sh in shapes:
                rs.tune_set_class(cls, knob, sh)

                def restore():
                    kb.copy_(k)
                    vb.copy_(v)
                g = rs.Graph(kb, vb if pairs else None)
                res[sh] = _time_graph(rs, torch, g, restore, reps)
                g.close()
            rs.tune_set_class(cls, knob, old)
            best[knob] = min(res, key=res.get)
            best[knob + "_ms"] = res
            rs.tune_set_class(cls, knob, best[knob])
        if n <= MSD_MAX_ITEMS:
            # MSD-first order (one top-digit pass + on-chip bucket sorts) or
            # the four LSD passes, with the chosen shapes; pairs + keys time.
            old_msd = rs.tune_get_class(cls, "msd")
            res = {}
            for msd in (0, 1):
                rs.tune_set_class(cls, "msd", msd)
                tot = 0.0
                for pairs in (True, False):
                    def restore():
                        kb.copy_(k)
                        vb.copy_(v)
                    g = rs.Graph(kb, vb if pairs else None)
                    tot += _time_graph(rs, torch, g, restore, reps)
                    g.close()
                res[msd] = tot
            rs.tune_set_class(cls, "msd", old_msd)
            best["msd"] = min(res, key=res.get)
            best["msd_ms"] = res
        if n >= DIGITS11_MIN_ITEMS:
            # Four 8-bit passes or three 11/11/10-bit ones (the graph's
            # workspace holds the latter's buffers when the class takes them).
            res = {}
            for digits in (8, 11):
                rs.tune_set_class(cls, "digits", digits)
                tot = 0.0
                for pairs in (True, False):
                    def restore():
                        kb.copy_(k)
                        vb.copy_(v)
                    g = rs.Graph(kb, vb if pairs else None)
                    tot += _time_graph(rs, torch, g, restore, reps)
                    g.close()
                res[digits] = tot
            best["digits"] = min(res, key=res.get)
            best["digits_ms"] = res
        for knob in ("tile_pairs", "tile_keys", "msd", "digits"):
            rs.tune_set_class(cls, knob, saved[knob])
        out[str(cls)] = best
        del k, v, kb, vb
        torch.cuda.empty_cache()
    return out


def tune_one_cta(rs, torch, inputs, reps=3):
    """Class 0 (up to 2^13 items): which whole arrays take the one-CTA sort
    (small_max 4096 or 8192; larger ones the scatter passes) and its digit
    width (4 or 8 bits), timed at 512 and at 8192 pairs; the score of a
    setting is the sum of its two times over the best ones."""
    cases = {}
    for n in (512, 8192):
        k = torch.from_numpy(inputs.keys("uniform", n, seed=300).view(np.int32)).cuda()
        v = torch.arange(n, dtype=torch.int32, device="cuda")
        cases[n] = (k, v, torch.empty_like(k), torch.empty_like(v))
    names = ("small_max", "small_bits")
    old = {k: rs.tune_get_class(0, k) for k in names}
    res = {}
    for small in (4096, 8192):
        for bits in (4, 8):
            for name, val in zip(names, (small, bits)):
                rs.tune_set_class(0, name, val)
            times = []
            for n, (k, v, kb, vb) in cases.items():
                def restore():
                    kb.copy_(k)
                    vb.copy_(v)
                g = rs.Graph(kb, vb)
                times.append(_time_graph(rs, torch, g, restore, reps))
                g.close()
            res["%d/%d" % (small, bits)] = times
    for name, val in old.items():
        rs.tune_set_class(0, name, val)
    best_t = [min(t[i] for t in res.values()) for i in range(2)]
    best = min(res, key=lambda c: sum(res[c][i] / best_t[i] for i in range(2)))
    small, bits = (int(x) for x in best.split("/"))
    return {"0": {"small_max": small, "small_bits": bits, "one_cta_ms": res}}


def tune_tiny_segments(rs, torch, inputs, reps=3):
    """Batches of 2^15 short arrays (sizes log-uniform on [2, 2^12]):
    one-warp sort threshold (0, 256 or 512) x digit width (4 or 8) for the
    size class of their average size."""
    k_np, v_np, off_np = inputs.segmented_batch(1 << 15, 1, 12, seed=11)
    cls = rs.size_class(k_np.size // (1 << 15))
    k = torch.from_numpy(k_np.view(np.int32)).cuda()
    v = torch.from_numpy(v_np.view(np.int32)).cuda()
    off = torch.from_numpy(off_np.view(np.int32)).cuda()
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    old = (rs.tune_get_class(cls, "warp_max"), rs.tune_get_class(cls, "small_bits"))
    res = {}
    for warp_max in (0, 256, 512):
        for bits in (4, 8):
            rs.tune_set_class(cls, "warp_max", warp_max)
            rs.tune_set_class(cls, "small_bits", bits)

            def restore():
                kb.copy_(k)
                vb.copy_(v)
            g = rs.Graph(kb, vb, off)
            res["%d/%d" % (warp_max, bits)] = _time_graph(rs, torch, g, restore, reps)
            g.close()
    rs.tune_set_class(cls, "warp_max", old[0])
    rs.tune_set_class(cls, "small_bits", old[1])
    best = min(res, key=res.get)
    warp_max, bits = (int(x) for x in best.split("/"))
    return {str(cls): {"warp_max": warp_max, "small_bits": bits, "tiny_segments_ms": res}}


def tune_segmented(rs, torch, inputs, reps=3, total=1 << 28):
    """Batches of 4096 arrays, sizes log-uniform on [2^8, 2^22], rescaled to
    `total` items; candidates: segmented tile shape x one-CTA threshold."""
    k_np, v_np, off_np = inputs.segmented_batch(4096, 8, 22, seed=10, scale_to=total)
    n = k_np.size
    cls = rs.size_class(n // 4096)
    k = torch.from_numpy(k_np.view(np.int32)).cuda()
    v = torch.from_numpy(v_np.view(np.int32)).cuda()
    off = torch.from_numpy(off_np.view(np.int32)).cuda()
    kb, vb = torch.empty_like(k), torch.empty_like(v)
    old = (rs.tune_get_class(cls, "tile_seg"), rs.tune_get_class(cls, "small_max"))
    res = {}
    for sh in range(len(rs.tile_shapes())):
        for small in (4096, 8192):
            rs.tune_set_class(cls, "tile_seg", sh)
            rs.tune_set_class(cls, "small_max", small)

            def restore():
                kb.copy_(k)
                vb.copy_(v)
            g = rs.Graph(kb, vb, off)
            res["%d/%d" % (sh, small)] = _time_graph(rs, torch, g, restore, reps)
            g.close()
    rs.tune_set_class(cls, "tile_seg", old[0])
    rs.tune_set_class(cls, "small_max", old[1])
    best = min(res, key=res.get)
    sh, small = (int(x) for x in best.split("/"))
    return {str(cls): {"tile_seg": sh, "small_max": small, "segmented_ms": res}}


def apply(table: dict) -> None:
    """Set the library's per-class knobs from a table made by this module."""
    from paper_1008_2849_gb300 import rs
    for cls, knobs in table.get("classes", {}).items():
        for name in ("tile_pairs", "tile_keys", "tile_seg", "small_max", "warp_max", "small_bits",
                     "msd", "digits"):
            if name in knobs:
                rs.tune_set_class(int(cls), name, int(knobs[name]))


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="tuning.json")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--quick", action="store_true", help="skip the 2^27 class")
    a = ap.parse_args(argv)
    import torch

    from paper_1008_2849_gb300 import build, inputs, rs
    build.build_library()
    rs.lib()
    classes = tune_whole(rs, torch, inputs, reps=a.reps, quick=a.quick)
    classes.update(tune_one_cta(rs, torch, inputs, reps=a.reps))
    for part in (tune_segmented(rs, torch, inputs, reps=a.reps),
                 tune_tiny_segments(rs, torch, inputs, reps=a.reps)):
        for cls, best in part.items():
            classes.setdefault(cls, {}).update(best)
    table = {"device": torch.cuda.get_device_name(0), "classes": classes}
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps({c: {k: v for k, v in d.items() if not k.endswith("_ms")}
                      for c, d in classes.items()}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
