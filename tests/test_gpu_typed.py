"""GPU parity tests of the typed-key sorts (signed 32-bit integers by value;
IEEE-754 binary32 by totalOrder) against the CPU oracle's typed sort, a
plain merge sort with the definitions' comparison, element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


def _golden_words():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "float_total_order.txt")
    return np.array([int(l.split("#", 1)[0].split()[0], 16) for l in open(path)
                     if l.split("#", 1)[0].strip()], dtype=np.uint32)


def _keys(kind, n, seed):
    if kind == "words":            # every bit pattern: NaNs, infinities, zeros of both signs
        return inputs.keys("uniform", n, seed)
    if kind == "specials":         # the totalOrder listing, many times over
        g = _golden_words()
        return g[inputs.splitmix32(seed, n, 0) % np.uint32(g.size)]
    if kind == "narrow":           # floats in [1, 2) differing in the low 16 bits only
        return np.uint32(0x3F800000) | (inputs.keys("uniform", n, seed) & np.uint32(0xFFFF))
    if kind == "small_ints":       # int32 in [-128, 127]
        u = (inputs.keys("uniform", n, seed) % np.uint32(256)).astype(np.int64)
        return (u - 128).astype(np.int32).view(np.uint32)
    if kind == "equal":
        return np.full(n, 0xBF800000, dtype=np.uint32)
    raise ValueError(kind)


def _check(rs, k, key_type, with_values=True):
    v = inputs.index_values(k.size) if with_values else None
    kd = to_dev(k)
    vd = to_dev(v) if with_values else None
    rs.sort_typed(kd, vd, key_type)
    ko, vo = oracle.sort_typed(k, v, key_type)
    assert np.array_equal(to_host(kd), ko)
    if with_values:
        assert np.array_equal(to_host(vd), vo)


SIZES = [1, 2, 100, 512, 513, 4096, 8192, 8193, 70_001, (1 << 20) + 37]


@pytest.mark.parametrize("key_type", ["i32", "f32"])
@pytest.mark.parametrize("n", SIZES)
def test_typed_sizes(rs, key_type, n):
    """Every path: one-warp, one-CTA and scatter-pass sorts, pairs and keys."""
    for kind in ("words", "specials"):
        k = _keys(kind, n, seed=120 + n % 97)
        _check(rs, k, key_type)
        _check(rs, k, key_type, with_values=False)


@pytest.mark.parametrize("kind,key_type", [("narrow", "f32"), ("small_ints", "i32"),
                                           ("equal", "f32"), ("specials", "i32")])
def test_typed_skipped_passes(rs, kind, key_type):
    """Keys whose mapped words share their top bytes (some passes are the
    identity and skipped, so the maps sit in passes other than 0 and 3) and
    all-equal keys (no pass moves data)."""
    k = _keys(kind, (1 << 20) + 3, seed=130)
    _check(rs, k, key_type)


@pytest.mark.parametrize("key_type", ["i32", "f32"])
def test_typed_segmented(rs, key_type):
    sizes = np.array([0, 1, 2, 300, 512, 513, 4096, 5000, 100_000, 33, 70_000, 0, 9000],
                     dtype=np.uint64)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1]) + 5
    for kind in ("words", "specials"):
        k = _keys(kind, n, seed=140)
        v = inputs.index_values(n)
        kd, vd, od = to_dev(k), to_dev(v), to_dev(off)
        rs.sort_typed(kd, vd, key_type, offsets=od)
        ko, vo = oracle.sort_typed_segmented(k, v, off, key_type)
        assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)


def test_typed_f32_2pow27_properties(rs):
    """2^27 float pairs of random bit patterns (scatter passes of the bench's
    size class): the output is a permutation, nondecreasing in totalOrder
    (checked through numpy's own encoding of the order), and stable."""
    n = 1 << 27
    k = inputs.keys("uniform", n, seed=150)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    rs.sort_typed(kd, vd, "f32")
    ko, vo = to_host(kd), to_host(vd)
    # totalOrder as a signed integer: flip the magnitude bits of negatives.
    s = ko.view(np.int32).astype(np.int64)
    ordered = np.where(s < 0, -(s & 0x7FFFFFFF) - 1, s)
    assert np.all(ordered[1:] >= ordered[:-1])
    assert np.array_equal(k[vo], ko)                      # value = input index
    same = ko[1:] == ko[:-1]
    assert np.all(vo[1:][same] > vo[:-1][same])           # stable
    assert np.array_equal(np.sort(vo), v)                 # permutation


def test_unknown_key_type_is_rejected(rs):
    import ctypes
    k = to_dev(inputs.keys("uniform", 100, seed=160))
    ws = rs.alloc_workspace(100, False)
    code = rs.lib().rs_sort_typed_ex(ctypes.c_void_p(k.data_ptr()), None, 100, 3, None,
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel())
    assert code == 1


@pytest.mark.parametrize("kind,key_type,n", [("words", "f32", 300_007), ("narrow", "f32", 70_001),
                                             ("small_ints", "i32", 1_000_003),
                                             ("words", "i32", 9000)])
def test_typed_one_or_two_instances(rs, kind, key_type, n):
    """Typed sorts with two scatter-pass instances per pass (the middle
    passes without the key map) and with one mapping instance per pass give
    the oracle's result either way, skipped passes included."""
    k = _keys(kind, n, seed=130)
    v = inputs.index_values(n)
    ko, vo = oracle.sort_typed(k, v, key_type)
    old = rs.tune_get("typed_split")
    try:
        for split_min in (0, 0x7FFFFFFF):
            rs.tune_set("typed_split", split_min)
            kd, vd = to_dev(k), to_dev(v)
            rs.sort_typed(kd, vd, key_type)
            assert np.array_equal(to_host(kd), ko), split_min
            assert np.array_equal(to_host(vd), vo), split_min
    finally:
        rs.tune_set("typed_split", old)
