"""CPU oracle for the stable LSD radix sort (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.

The arithmetic lives in ``rs_oracle.c`` (plain C, compiled here with gcc into
``liboracle.so``); this module only marshals numpy arrays across ctypes.
Every function follows the paper's definitions:

* ``digit_histograms`` / ``exclusive_prefix`` -- counting and prefix-sum steps
  of the naive counting sort (Sec. 3; Alg. 2 ``PrefixSum``).
* ``counting_pass`` -- one stable counting-sort pass by byte ``p`` (Sec. 3).
* ``sort_pairs`` / ``sort_keys`` -- LSD radix sort, K = 32, D = 8, four
  passes (Sec. 4).
* ``sort_pairs_segmented`` -- the same sort inside every segment (no paper
  counterpart; plain definition).
* ``sort_pairs_threaded`` -- same result on several host threads, used to time
  the CPU baseline.
* ``sort_pairs64`` -- the LSD radix sort of 64-bit keys (K = 64, D = 8: eight
  passes), optionally carrying 32-bit values.
* ``sort_typed`` / ``sort_typed_segmented`` -- stable sorts of signed 32-bit
  integer keys (by value) and of IEEE-754 binary32 keys (by the totalOrder
  predicate of IEEE 754-2008 Sec. 5.10): no paper counterpart; a plain merge
  sort with that comparison.
* ``sort_kv`` -- keys and values of every width (Sec. 1: larger items sort
  the same way): 32-bit or 64-bit keys, unsigned, signed or IEEE float, with
  no, 32-bit or 64-bit values; a plain stable merge sort by the key.

Every function takes an optional ``lib`` (a library bound by ``_bind``) so that
the pin tests can also be run against deliberately mutated builds of the C
source, to show that the pins catch plausible mistakes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile ``rs_oracle.c`` into ``liboracle.so`` (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.oracle_digit_histograms.argtypes = [_u32p, ctypes.c_size_t, _u64p]
    lib.oracle_digit_histograms.restype = None
    lib.oracle_exclusive_prefix.argtypes = [_u64p, _u64p]
    lib.oracle_exclusive_prefix.restype = None
    lib.oracle_counting_pass.argtypes = [_u32p, _u32p, _u32p, _u32p,
                                         ctypes.c_size_t, ctypes.c_uint]
    lib.oracle_counting_pass.restype = None
    lib.oracle_sort_pairs.argtypes = [_u32p, _u32p, _u32p, _u32p, ctypes.c_size_t]
    lib.oracle_sort_pairs.restype = ctypes.c_int
    lib.oracle_sort_pairs_segmented.argtypes = [_u32p, _u32p, _u32p, _u32p,
                                                ctypes.c_size_t, _u32p, ctypes.c_uint32]
    lib.oracle_sort_pairs_segmented.restype = ctypes.c_int
    lib.oracle_sort_pairs_threaded.argtypes = [_u32p, _u32p, _u32p, _u32p,
                                               ctypes.c_size_t, ctypes.c_uint]
    lib.oracle_sort_pairs_threaded.restype = ctypes.c_int
    if hasattr(lib, "oracle_sort_pairs64"):
        lib.oracle_sort_pairs64.argtypes = [_u64p, _u32p, _u64p, _u32p, ctypes.c_size_t]
        lib.oracle_sort_pairs64.restype = ctypes.c_int
    if hasattr(lib, "oracle_sort_typed"):  # mutated copies of older sources lack it
        lib.oracle_sort_typed.argtypes = [_u32p, _u32p, _u32p, _u32p, ctypes.c_size_t,
                                          ctypes.c_int]
        lib.oracle_sort_typed.restype = ctypes.c_int
        lib.oracle_sort_typed_segmented.argtypes = [_u32p, _u32p, _u32p, _u32p, ctypes.c_size_t,
                                                    _u32p, ctypes.c_uint32, ctypes.c_int]
        lib.oracle_sort_typed_segmented.restype = ctypes.c_int
    if hasattr(lib, "oracle_sort_kv"):
        lib.oracle_sort_kv.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                       ctypes.c_int]
        lib.oracle_sort_kv.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _u32(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint32:
        raise TypeError("expected uint32 array, got %s" % a.dtype)
    return a


def _ptr(a, kind=_u32p):
    return None if a is None else a.ctypes.data_as(kind)


def digit_histograms(keys, lib=None) -> np.ndarray:
    """H[p, b] = number of keys whose byte p equals b; shape (4, 256), uint64."""
    keys = _u32(keys)
    h = np.zeros((4, 256), dtype=np.uint64)
    (lib or _load()).oracle_digit_histograms(_ptr(keys), keys.size, _ptr(h, _u64p))
    return h


def exclusive_prefix(hist, lib=None) -> np.ndarray:
    """G[p, b] = sum of H[p, b'] over b' < b; shape (4, 256), uint64."""
    h = np.ascontiguousarray(hist, dtype=np.uint64).reshape(4, 256)
    g = np.zeros((4, 256), dtype=np.uint64)
    (lib or _load()).oracle_exclusive_prefix(_ptr(h, _u64p), _ptr(g, _u64p))
    return g


def counting_pass(keys, vals, p: int, lib=None):
    """One stable counting-sort pass by byte ``p``; returns (keys, vals|None)."""
    keys = _u32(keys)
    vals = None if vals is None else _u32(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    (lib or _load()).oracle_counting_pass(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.size, p)
    return ko, vo


def sort_pairs(keys, vals, lib=None):
    """Stable ascending LSD radix sort; returns new (keys, vals) arrays."""
    keys = _u32(keys)
    vals = None if vals is None else _u32(vals)
    if vals is not None and vals.size != keys.size:
        raise ValueError("keys and vals differ in length")
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_pairs(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.size)
    if rc:
        raise MemoryError("oracle_sort_pairs failed (%d)" % rc)
    return ko, vo


def sort_keys(keys, lib=None) -> np.ndarray:
    return sort_pairs(keys, None, lib)[0]


def sort_pairs_segmented(keys, vals, offsets, lib=None):
    """Sort every segment [offsets[s], offsets[s+1]) on its own."""
    keys = _u32(keys)
    vals = None if vals is None else _u32(vals)
    offsets = _u32(offsets)
    nseg = max(offsets.size - 1, 0)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_pairs_segmented(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo),
                                             keys.size, _ptr(offsets), nseg)
    if rc == -2:
        raise ValueError("malformed segment table")
    if rc:
        raise MemoryError("oracle_sort_pairs_segmented failed (%d)" % rc)
    return ko, vo


def sort_pairs_threaded(keys, vals, nthreads: int, lib=None):
    """Same result as ``sort_pairs`` computed by ``nthreads`` host threads."""
    keys = _u32(keys)
    vals = None if vals is None else _u32(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_pairs_threaded(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo),
                                            keys.size, int(nthreads))
    if rc:
        raise MemoryError("oracle_sort_pairs_threaded failed (%d)" % rc)
    return ko, vo


KEY_TYPES = {"u32": 0, "i32": 1, "f32": 2}
# Every key type of sort_kv: (code, word dtype).
KV_KEY_TYPES = {"u32": (0, np.uint32), "i32": (1, np.uint32), "f32": (2, np.uint32),
                "u64": (3, np.uint64), "i64": (4, np.uint64), "f64": (5, np.uint64)}


def sort_typed(keys, vals, key_type: str, lib=None):
    """Stable ascending sort of 32-bit keys read as ``key_type`` ("u32",
    "i32" or "f32", given as uint32 bit patterns); returns (keys, vals|None)."""
    keys = _u32(keys)
    vals = None if vals is None else _u32(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_typed(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.size,
                                            KEY_TYPES[key_type])
    if rc:
        raise MemoryError("oracle_sort_typed failed (%d)" % rc)
    return ko, vo


def sort_typed_segmented(keys, vals, offsets, key_type: str, lib=None):
    """``sort_typed`` inside every segment [offsets[s], offsets[s+1])."""
    keys = _u32(keys)
    vals = None if vals is None else _u32(vals)
    offsets = _u32(offsets)
    nseg = max(offsets.size - 1, 0)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_typed_segmented(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo),
                                                      keys.size, _ptr(offsets), nseg,
                                                      KEY_TYPES[key_type])
    if rc == -2:
        raise ValueError("malformed segment table")
    if rc:
        raise MemoryError("oracle_sort_typed_segmented failed (%d)" % rc)
    return ko, vo


def sort_pairs64(keys, vals, lib=None):
    """Stable ascending LSD radix sort of uint64 keys (eight 8-bit passes),
    values uint32 or None; returns new (keys, vals) arrays."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype != np.uint64:
        raise TypeError("expected uint64 keys, got %s" % keys.dtype)
    vals = None if vals is None else _u32(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_pairs64(_ptr(keys, _u64p), _ptr(vals), _ptr(ko, _u64p),
                                              _ptr(vo), keys.size)
    if rc:
        raise MemoryError("oracle_sort_pairs64 failed (%d)" % rc)
    return ko, vo


def sort_kv(keys, vals, key_type: str, lib=None):
    """Stable ascending sort of keys read as ``key_type`` (one of
    ``KV_KEY_TYPES``; bit patterns as uint32 or uint64 words), carrying
    ``vals`` (uint32, uint64 or None) as opaque payloads; returns new
    (keys, vals|None) arrays."""
    code, kdt = KV_KEY_TYPES[key_type]
    keys = np.ascontiguousarray(keys)
    if keys.dtype != kdt:
        raise TypeError("expected %s keys for %s, got %s" % (np.dtype(kdt), key_type, keys.dtype))
    value_bits = 0
    if vals is not None:
        vals = np.ascontiguousarray(vals)
        if vals.dtype not in (np.uint32, np.uint64) or vals.size != keys.size:
            raise TypeError("values must be uint32 or uint64, one per key")
        value_bits = 8 * vals.dtype.itemsize
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = (lib or _load()).oracle_sort_kv(keys.ctypes.data, None if vals is None else vals.ctypes.data,
                                         ko.ctypes.data, None if vo is None else vo.ctypes.data,
                                         keys.size, code, value_bits)
    if rc:
        raise MemoryError("oracle_sort_kv failed (%d)" % rc)
    return ko, vo


def sort_kv_segmented(keys, vals, offsets, key_type: str, lib=None):
    """``sort_kv`` inside every segment [offsets[s], offsets[s+1]): the
    definition of the segmented sort, one segment at a time; items outside
    [offsets[0], offsets[-1]) are copied unchanged.  Returns new arrays."""
    offsets = np.asarray(offsets, dtype=np.int64)
    if offsets.size and (np.any(np.diff(offsets) < 0) or offsets[0] < 0
                         or offsets[-1] > np.asarray(keys).size):
        raise ValueError("malformed segment table")
    ko = np.array(keys, copy=True)
    vo = None if vals is None else np.array(vals, copy=True)
    for a, b in zip(offsets[:-1], offsets[1:]):
        if b - a < 2:
            continue
        sk, sv = sort_kv(ko[a:b], None if vo is None else vo[a:b], key_type, lib=lib)
        ko[a:b] = sk
        if vo is not None:
            vo[a:b] = sv
    return ko, vo
