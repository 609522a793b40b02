"""GPU parity tests of the sorts of every item width (rs_sort_kv_ex): 32-bit
and 64-bit keys, unsigned, signed or IEEE float, carrying no, 32-bit or 64-bit
values, against the CPU oracle's plain stable merge sort (oracle.sort_kv),
element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs

pytestmark = pytest.mark.gpu

KEY_TYPES = ["u32", "i32", "f32", "u64", "i64", "f64"]


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


def _golden(name, dtype):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    return np.array([int(l.split("#", 1)[0].split()[0], 16) for l in open(path)
                     if l.split("#", 1)[0].strip()], dtype=dtype)


def _keys(key_type, kind, n, seed):
    wide = key_type.endswith("64")
    lo = inputs.splitmix32(seed, n, 0)
    if not wide:
        if kind == "words":
            return lo
        if kind == "specials":
            g = _golden("float_total_order.txt", np.uint32)
            return g[lo % np.uint32(g.size)]
        if kind == "narrow":       # shared top bytes: the maps sit in passes 0 and 1
            return np.uint32(0x3F800000) | (lo & np.uint32(0xFFFF))
        if kind == "equal":
            return np.full(n, 0xBF800000, dtype=np.uint32)
    hi = inputs.splitmix32(seed, n, 1).astype(np.uint64)
    if kind == "words":            # every bit pattern: NaNs, infinities, zeros, extremes
        return (hi << np.uint64(32)) | lo.astype(np.uint64)
    if kind == "specials":
        g = _golden("double_total_order.txt", np.uint64)
        return g[lo % np.uint32(g.size)]
    if kind == "narrow":           # binary64 in [1, 2) differing in the low 16 bits
        return np.uint64(0x3FF0000000000000) | (lo & np.uint32(0xFFFF)).astype(np.uint64)
    if kind == "equal":
        return np.full(n, 0xBFF0000000000000, dtype=np.uint64)
    raise ValueError(kind)


def _values(value_bits, n):
    if value_bits == 0:
        return None
    i = np.arange(n, dtype=np.uint64)
    if value_bits == 32:
        return i.astype(np.uint32)
    return (i ^ np.uint64(0xA5A5A5A5)) << np.uint64(32) | i   # halves differ


def _dev(a):
    import torch
    if a is None:
        return None
    return torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32)).cuda()


def _host(t, like):
    return t.cpu().numpy().view(like.dtype)


def _check(rs, k, key_type, value_bits):
    v = _values(value_bits, k.size)
    kd, vd = _dev(k), _dev(v)
    rs.sort_kv(kd, vd, key_type)
    ko, vo = oracle.sort_kv(k, v, key_type)
    assert np.array_equal(_host(kd, k), ko)
    if v is not None:
        assert np.array_equal(_host(vd, v), vo)


SIZES = [1, 2, 100, 2304, 2305, 2688, 2689, 70_001, (1 << 20) + 37]


@pytest.mark.parametrize("value_bits", [0, 32, 64])
@pytest.mark.parametrize("key_type", KEY_TYPES)
@pytest.mark.parametrize("n", SIZES)
def test_kv_sizes(rs, n, key_type, value_bits):
    """One partial tile, exactly one wide tile (384 x 6 and 384 x 7), one
    more, several tiles with a ragged tail; random words of every pattern."""
    _check(rs, _keys(key_type, "words", n, seed=200 + n % 89), key_type, value_bits)


@pytest.mark.parametrize("kind", ["specials", "narrow", "equal"])
@pytest.mark.parametrize("key_type", KEY_TYPES)
def test_kv_distributions(rs, key_type, kind):
    """The totalOrder listings many times over (NaNs of both signs, -0, +0,
    subnormals), keys sharing their top bytes (skipped passes: the maps sit in
    the passes that execute) and all keys equal (no pass moves data), with
    64-bit values."""
    _check(rs, _keys(key_type, kind, (1 << 20) + 3, seed=210), key_type, 64)


def test_kv_u64_matches_sort64(rs):
    """rs_sort64_ex is the unsigned 64-bit case of rs_sort_kv_ex."""
    k = _keys("u64", "words", 300_001, seed=220)
    v = _values(32, k.size)
    a_k, a_v, b_k, b_v = _dev(k), _dev(v), _dev(k), _dev(v)
    rs.sort64(a_k, a_v)
    rs.sort_kv(b_k, b_v, "u64")
    assert np.array_equal(_host(a_k, k), _host(b_k, k))
    assert np.array_equal(_host(a_v, v), _host(b_v, v))


@pytest.mark.parametrize("key_type", ["u32", "f64"])
def test_kv_v64_2pow27_properties(rs, key_type):
    """2^27 items with 64-bit values at full size: keys nondecreasing in the
    typed order (numpy's reading of the words, no NaNs drawn), each value
    still with its key, and equal keys in input order."""
    n = 1 << 27
    k = _keys(key_type, "words", n, seed=230)
    if key_type == "f64":          # clear NaN exponents so numpy can order the words
        nan = (k & np.uint64(0x7FF0000000000000)) == np.uint64(0x7FF0000000000000)
        k[nan] &= np.uint64(0xBFFFFFFFFFFFFFFF)
    v = _values(64, n)
    kd, vd = _dev(k), _dev(v)
    rs.sort_kv(kd, vd, key_type)
    ko, vo = _host(kd, k), _host(vd, v)
    idx = (vo & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(vo, v[idx])                      # whole values, a permutation
    assert np.array_equal(np.sort(idx), np.arange(n))
    assert np.array_equal(ko, k[idx])                      # each key with its value
    view = ko.view(np.float64) if key_type == "f64" else ko
    d = np.diff(view)
    assert np.all(d >= 0)
    same = ko[1:] == ko[:-1]
    assert np.all(idx[1:][same] > idx[:-1][same])          # stable


def test_kv_argument_errors(rs):
    import ctypes
    import torch
    k = torch.zeros(16, dtype=torch.int64, device="cuda")
    v = torch.zeros(16, dtype=torch.int64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    L = rs.lib()
    w = ctypes.c_void_p(ws.data_ptr())
    assert L.rs_sort_kv_ex(ctypes.c_void_p(k.data_ptr() + 4), ctypes.c_void_p(v.data_ptr()), 8,
                           3, 64, None, w, ws.numel()) == 1        # misaligned 64-bit keys
    assert L.rs_sort_kv_ex(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr() + 4), 8,
                           0, 64, None, w, ws.numel()) == 1        # misaligned 64-bit values
    assert L.rs_sort_kv_ex(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr()), 16,
                           4, 64, None, w, 16) == 1                # workspace too small
    assert L.rs_sort_kv_ex(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(k.data_ptr() + 32), 8,
                           5, 64, None, w, ws.numel()) == 1        # overlapping
