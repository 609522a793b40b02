"""CPU-only tests of the per-size-class tuning table (host settings only)."""
from __future__ import annotations

import json
import os

import pytest


@pytest.fixture(scope="module")
def rs():
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


def test_size_classes(rs):
    assert rs.size_class(1) == 0 and rs.size_class(8192) == 0
    assert rs.size_class(8193) == 1 and rs.size_class(1 << 16) == 1
    assert rs.size_class((1 << 20) + 1) == 3
    assert rs.size_class(1 << 28) == 4 and rs.size_class((1 << 28) + 1) == 5


def test_apply_table_and_restore(rs, tmp_path):
    from paper_1008_2849_gb300 import autotune
    saved = {(c, k): rs.tune_get_class(c, k) for c in range(6)
             for k in ("tile_pairs", "tile_keys", "tile_seg", "small_max", "digits")}
    try:
        table = {"device": "test", "classes": {"2": {"tile_pairs": 1, "tile_keys": 2},
                                               "4": {"tile_seg": 5, "small_max": 8192,
                                                     "digits": 11}}}
        p = tmp_path / "t.json"
        p.write_text(json.dumps(table))
        autotune.apply(autotune.load(str(p)))
        assert rs.tune_get_class(2, "tile_pairs") == 1 and rs.tune_get_class(2, "tile_keys") == 2
        assert rs.tune_get_class(4, "tile_seg") == 5 and rs.tune_get_class(4, "small_max") == 8192
        assert rs.tune_get_class(4, "digits") == 11 and rs.tune_get_class(3, "digits") == 8
        assert rs.tune_get_class(3, "tile_pairs") == saved[(3, "tile_pairs")]
        with pytest.raises(rs.RsError):
            rs.tune_set_class(0, "tile_pairs", 99)
        with pytest.raises(rs.RsError):
            rs.tune_set_class(7, "tile_pairs", 0)
    finally:
        for (c, k), v in saved.items():
            rs.tune_set_class(c, k, v)


def test_committed_table_applies(rs):
    """The measured GB300 table loads and applies; it keeps 8-bit digits and
    the one-CTA sort limits within range."""
    import os
    from paper_1008_2849_gb300 import autotune
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    table = autotune.load(os.path.join(root, "paper_1008_2849_gb300", "tuning_gb300.json"))
    saved = {(c, k): rs.tune_get_class(c, k) for c in range(6)
             for k in ("tile_pairs", "tile_keys", "tile_seg", "small_max", "warp_max",
                       "small_bits", "msd", "digits")}
    try:
        autotune.apply(table)
        for c in range(6):
            assert rs.tune_get_class(c, "digits") == 8
            assert 0 <= rs.tune_get_class(c, "small_max") <= 8192
    finally:
        for (c, k), v in saved.items():
            rs.tune_set_class(c, k, v)


def test_device_generator_matches_numpy_on_cpu():
    """The torch generator (used to draw serving workloads on the GPU) gives
    the same words as the numpy one; checked with torch's CPU backend."""
    import numpy as np
    import torch

    from paper_1008_2849_gb300 import inputs
    for seed, n, start in ((11, 1000, 0), (12345, 70001, 5), (3, 1, 1 << 40)):
        a = inputs.splitmix32(seed, n, 0, start=start)
        b = inputs.splitmix32_torch(seed, n, 0, start=start, device="cpu").numpy().view(np.uint32)
        assert np.array_equal(a, b)
    for dist in ("uniform", "and2"):
        a = inputs.keys(dist, 5000, 77)
        b = inputs.keys_torch(dist, 5000, 77, device="cpu").numpy().view(np.uint32)
        assert np.array_equal(a, b), dist


def test_knob_table_matches_header(rs):
    """Every RS_TUNE_* value of include/rs.h has the same number in the binding."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "rs.h")).read()
    header = {m.group(1).lower(): int(m.group(2))
              for m in re.finditer(r"RS_TUNE_([A-Z0-9_]+)\s*=\s*(\d+)", text)}
    assert header == rs.TUNE_KNOBS


def test_on_chip_sort_knobs_are_checked(rs):
    saved = [(c, k, rs.tune_get_class(c, k)) for c in range(6) for k in ("warp_max", "small_bits")]
    try:
        for bits in (4, 8):
            rs.tune_set_class(1, "small_bits", bits)
            assert rs.tune_get_class(1, "small_bits") == bits
        for bad in (0, 5, 16):
            with pytest.raises(rs.RsError):
                rs.tune_set_class(1, "small_bits", bad)
        rs.tune_set_class(1, "warp_max", 512)
        rs.tune_set_class(1, "warp_max", 0)
        assert rs.tune_get_class(1, "warp_max") == 0
        with pytest.raises(rs.RsError):
            rs.tune_set_class(1, "warp_max", 513)
    finally:
        for c, k, v in saved:
            rs.tune_set_class(c, k, v)


def test_digits_knob_sizes_the_workspace(rs):
    """RS_TUNE_DIGITS = 11 in a size class makes rs_workspace_bytes cover the
    11-bit order's buffers for that class only; 8 restores the 8-bit size."""
    n4, n3 = 1 << 26, 1 << 22  # classes 4 and 3
    base4, base3 = rs.workspace_bytes(n4, True), rs.workspace_bytes(n3, True)
    old = rs.tune_get_class(4, "digits")
    assert old == 8
    try:
        rs.tune_set_class(4, "digits", 11)
        assert rs.workspace_bytes(n4, True) == max(base4, rs.workspace_bytes_digits11(n4, True))
        assert rs.workspace_bytes(n4, True) > base4
        assert rs.workspace_bytes(n3, True) == base3
        for bad in (0, 4, 9, 12):
            with pytest.raises(rs.RsError):
                rs.tune_set_class(4, "digits", bad)
    finally:
        rs.tune_set_class(4, "digits", old)
    assert rs.workspace_bytes(n4, True) == base4
    assert rs.tune_get("d11_shape") == 1
    for bad in (-1, 4):
        with pytest.raises(rs.RsError):
            rs.tune_set("d11_shape", bad)


def test_traffic_record_follows_the_kernel_source(tmp_path):
    """bench.py's recorded ncu traffic is used only while the scatter kernel's
    code is the code it was captured from: comment edits and unrelated header
    lines keep the source hash, code and tile-shape edits change it; the
    committed record matches the current sources."""
    import shutil
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    assert bench.recorded_traffic() is not None
    for p in bench.ONESWEEP_SOURCES:
        path = p.split(":")[0]
        (tmp_path / os.path.dirname(path)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(root, path), tmp_path / path)
    old_root = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        base = bench.source_hash(bench.ONESWEEP_SOURCES)
        hdr = tmp_path / "paper_1008_2849_gb300/csrc/rs_internal.h"
        kern = tmp_path / "paper_1008_2849_gb300/csrc/rs_onesweep.cuh"
        text_h, text_k = hdr.read_text(), kern.read_text()
        hdr.write_text(text_h + "\n// a comment\nconstexpr int kUnrelated = 3;\n")
        kern.write_text(text_k.replace("#pragma once", "#pragma once  // a comment", 1))
        assert bench.source_hash(bench.ONESWEEP_SOURCES) == base
        hdr.write_text(text_h.replace("X(3, 384, 13, 2, 6)", "X(3, 384, 12, 2, 6)"))
        assert bench.source_hash(bench.ONESWEEP_SOURCES) != base
        hdr.write_text(text_h)
        kern.write_text(text_k.replace("#pragma once", "#pragma once\nstatic int x_;", 1))
        assert bench.source_hash(bench.ONESWEEP_SOURCES) != base
    finally:
        bench.ROOT = old_root
