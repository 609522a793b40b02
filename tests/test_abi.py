"""CPU-only checks of the C ABI: the library builds, loads without a GPU,
exports every entry point include/rs.h declares, and rejects bad arguments
on the host before touching CUDA."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(rs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1008_2849_gb300 import build, rs
    build.build_library()
    return rs.lib()


def test_header_declares_core_calls():
    names = header_functions()
    for must in ("rs_sort_keys", "rs_sort_pairs", "rs_sort_keys_ex", "rs_sort_pairs_ex",
                 "rs_workspace_bytes", "rs_stream_status", "rs_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), "librs.so does not export %s" % name


def test_binding_covers_header():
    from paper_1008_2849_gb300 import rs
    assert sorted(rs.SIGNATURES) == header_functions()


def test_status_strings(lib):
    from paper_1008_2849_gb300 import rs
    for code in range(0, 8):
        s = rs.status_string(code)
        assert s and s != "unknown status"
    assert rs.status_string(99) == "unknown status"


def test_workspace_bytes(lib):
    from paper_1008_2849_gb300 import rs
    assert rs.workspace_bytes(0, True) == 0
    small = rs.workspace_bytes(1000, False)
    pairs = rs.workspace_bytes(1000, True)
    assert pairs > small > 0
    n = 1 << 28
    ws = rs.workspace_bytes(n, True)
    # alternate key and value buffers plus look-back status and control
    # at most two status arrays of 1 KiB per 4096-item tile, plus 64 KiB
    assert 8 * n <= ws <= 8 * n + 2 * (n // 4096) * 1024 + 65536
    assert ws % 256 == 0


def test_host_side_argument_errors(lib):
    from paper_1008_2849_gb300 import rs
    # All of these are rejected before any CUDA call.
    assert lib.rs_sort_keys(None, 5) == 1                  # null keys
    assert lib.rs_sort_pairs(ctypes.c_void_p(4096), None, 5) == 1   # null values
    assert lib.rs_sort_keys(ctypes.c_void_p(4096), 1 << 32) == 5    # n >= 2^32
    assert lib.rs_sort_keys(ctypes.c_void_p(4098), 5) == 1          # misaligned
    # keys and values overlap
    assert lib.rs_sort_pairs(ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 8), 5) == 1
    # n = 0 is a no-op
    assert lib.rs_sort_keys(None, 0) == 0
    assert lib.rs_sort_pairs_ex(ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20), 100, None, None, 0) == 1
    assert lib.rs_digit_histograms_ex(ctypes.c_void_p(4096), 10, None, None) == 1
    assert lib.rs_sort_pairs_host(None, None, None, None, 10) == 1
    assert lib.rs_sort_pairs_host_batch(None, None, None, None, None, 0) == 0   # nothing to do
    assert lib.rs_sort_pairs_host_batch(None, None, None, None, None, 2) == 1   # no tables
    P = ctypes.c_void_p * 2
    tab = P(4096, None)
    sizes = (ctypes.c_size_t * 2)(10, 10)
    assert lib.rs_sort_pairs_host_batch(tab, None, tab, None, sizes, 2) == 1   # a NULL entry
    big = (ctypes.c_size_t * 2)(1 << 32, 0)
    assert lib.rs_sort_pairs_host_batch(tab, None, tab, None, big, 2) == 5     # n >= 2^32


def test_workspace_bytes_digits11(lib):
    from paper_1008_2849_gb300 import rs
    assert rs.workspace_bytes_digits11(0, True) == 0
    assert rs.workspace_bytes_digits11(1 << 32, True) == 0
    for n in (1, 4095, 4097, 1_000_003, 1 << 28):
        keys_only = rs.workspace_bytes_digits11(n, False)
        pairs = rs.workspace_bytes_digits11(n, True)
        # two alternate key (and value) buffers, per-chunk counts of at most
        # 1024 chunks of 2048 buckets, the bucket totals, 256-byte rounding
        assert 8 * n <= keys_only <= 8 * n + 1024 * 2048 * 4 + 8192 + 1024
        assert 16 * n <= pairs <= 16 * n + 1024 * 2048 * 4 + 8192 + 2048
        assert keys_only % 256 == 0 and pairs % 256 == 0
    # Host-side refusals, before any CUDA call.
    assert lib.rs_sort_digits11_ex(None, None, 5, None, ctypes.c_void_p(4096), 1 << 20) == 1
    assert lib.rs_sort_digits11_ex(ctypes.c_void_p(4096), None, 100, None, None, 0) == 1
    assert lib.rs_sort_digits11_ex(ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 8), 100, None,
                                   ctypes.c_void_p(1 << 20), 1 << 20) == 1     # overlap
    assert lib.rs_sort_digits11_ex(ctypes.c_void_p(4096), None, 1 << 32, None,
                                   ctypes.c_void_p(1 << 20), 1 << 20) == 5     # n >= 2^32
    assert lib.rs_sort_digits11_ex(ctypes.c_void_p(4096), None, 100, None,
                                   ctypes.c_void_p(1 << 20), 16) == 1          # too small
    assert lib.rs_sort_digits11_ex(None, None, 0, None, None, 0) == 0          # nothing to do


def test_workspace_bytes_kv(lib):
    from paper_1008_2849_gb300 import rs
    n = 1 << 20
    # 32-bit keys with no or 32-bit values: the workspace of the 32-bit sorts.
    assert rs.workspace_bytes_kv(n, "u32", 0) == rs.workspace_bytes(n, False)
    assert rs.workspace_bytes_kv(n, "f32", 32) == rs.workspace_bytes(n, True)
    assert rs.workspace_bytes_kv(n, "u64", 32) == rs.workspace_bytes64(n, True)
    assert rs.workspace_bytes_kv(n, "i64", 0) == rs.workspace_bytes64(n, False)
    # Wide items: alternate key and value buffers plus two status arrays of
    # 1 KiB per tile (2304 items at least) and the control block.
    for kt, kb in (("u32", 4), ("u64", 8), ("f64", 8)):
        ws = rs.workspace_bytes_kv(n, kt, 64)
        assert (kb + 8) * n <= ws <= (kb + 8) * n + 2 * (n // 2304 + 1) * 1024 + 65536
        assert ws % 256 == 0
    assert rs.workspace_bytes_kv(0, "u64", 64) == 0
    assert lib.rs_workspace_bytes_kv(100, 6, 0) == 0      # unknown key type
    assert lib.rs_workspace_bytes_kv(100, 3, 16) == 0     # unknown value width


def test_kv_host_side_argument_errors(lib):
    k, v, ws = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 30), ctypes.c_void_p(1 << 34)
    big = 1 << 40
    assert lib.rs_sort_kv_ex(k, v, 100, 6, 64, None, ws, big) == 1           # key type
    assert lib.rs_sort_kv_ex(k, v, 100, 3, 16, None, ws, big) == 1           # value width
    assert lib.rs_sort_kv_ex(k, None, 100, 3, 64, None, ws, big) == 1        # values missing
    assert lib.rs_sort_kv_ex(k, v, 100, 3, 0, None, ws, big) == 1            # values unexpected
    assert lib.rs_sort_kv_ex(ctypes.c_void_p((1 << 20) + 4), v, 100, 3, 64, None, ws, big) == 1
    assert lib.rs_sort_kv_ex(k, ctypes.c_void_p((1 << 30) + 4), 100, 0, 64, None, ws, big) == 1
    assert lib.rs_sort_kv_ex(k, ctypes.c_void_p((1 << 20) + 512), 100, 3, 64, None, ws, big) == 1
    assert lib.rs_sort_kv_ex(k, v, 100, 4, 64, None, None, 0) == 1           # no workspace
    assert lib.rs_sort_kv_ex(k, v, 100, 4, 64, None, ws, 64) == 1            # too small
    assert lib.rs_sort_kv_ex(k, v, 1 << 32, 4, 64, None, ws, big) == 5       # n >= 2^32
    assert lib.rs_sort_kv_ex(None, None, 0, 5, 0, None, None, 0) == 0        # n = 0
