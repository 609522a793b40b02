"""Python binding of librs.so (argument marshalling only).

Every function here forwards to the extern "C" entry point of the same name
in ``include/rs.h``; the sort runs entirely in the library's CUDA kernels.
PyTorch only supplies device memory and streams: tensors are passed as raw
device pointers (``data_ptr()``) and the current stream's handle.  There is
no fallback: if ``librs.so`` is missing or no sm_103a GPU is present, the
calls raise.

Tensors must be contiguous CUDA tensors of 4-byte elements (``torch.int32``
or ``torch.uint32``); int32 tensors are read as their unsigned bit patterns.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librs.so")

RS_OK = 0
STATUS_NAMES = {0: "RS_OK", 1: "RS_ERR_INVALID_ARG", 2: "RS_ERR_OUT_OF_MEMORY", 3: "RS_ERR_CUDA",
                4: "RS_ERR_TIMEOUT", 5: "RS_ERR_UNSUPPORTED", 6: "RS_ERR_BOUNDS",
                7: "RS_ERR_BAD_SEGMENTS"}

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_u32 = ctypes.c_uint32
_int = ctypes.c_int

# name -> (restype, argtypes); mirrors include/rs.h
SIGNATURES = {
    "rs_sort_keys": (_int, [_vp, _sz]),
    "rs_sort_pairs": (_int, [_vp, _vp, _sz]),
    "rs_sort_keys_ex": (_int, [_vp, _sz, _vp, _vp, _sz]),
    "rs_sort_pairs_ex": (_int, [_vp, _vp, _sz, _vp, _vp, _sz]),
    "rs_sort_digits11_ex": (_int, [_vp, _vp, _sz, _vp, _vp, _sz]),
    "rs_workspace_bytes_digits11": (_sz, [_sz, _int]),
    "rs_sort_keys_segmented": (_int, [_vp, _sz, _vp, _u32]),
    "rs_sort_pairs_segmented": (_int, [_vp, _vp, _sz, _vp, _u32]),
    "rs_sort_keys_segmented_ex": (_int, [_vp, _sz, _vp, _u32, _vp, _vp, _sz]),
    "rs_sort_pairs_segmented_ex": (_int, [_vp, _vp, _sz, _vp, _u32, _vp, _vp, _sz]),
    "rs_sort_typed_ex": (_int, [_vp, _vp, _sz, _int, _vp, _vp, _sz]),
    "rs_sort_segmented_typed_ex": (_int, [_vp, _vp, _sz, _vp, _u32, _int, _vp, _vp, _sz]),
    "rs_workspace_bytes": (_sz, [_sz, _int, _u32]),
    "rs_sort64_ex": (_int, [_vp, _vp, _sz, _vp, _vp, _sz]),
    "rs_workspace_bytes64": (_sz, [_sz, _int]),
    "rs_sort_kv_ex": (_int, [_vp, _vp, _sz, _int, _int, _vp, _vp, _sz]),
    "rs_workspace_bytes_kv": (_sz, [_sz, _int, _int]),
    "rs_sort_kv_segmented_ex": (_int, [_vp, _vp, _sz, _vp, _u32, _int, _int, _vp, _vp, _sz]),
    "rs_workspace_bytes_kv_segmented": (_sz, [_sz, _int, _int, _u32]),
    "rs_stream_status": (_int, [_vp]),
    "rs_status_string": (ctypes.c_char_p, [_int]),
    "rs_digit_histograms_ex": (_int, [_vp, _sz, _vp, _vp]),
    "rs_msd_partition_ex": (_int, [_vp, _vp, _sz, _vp, _vp, _vp, _vp, _vp, _sz]),
    "rs_sort_pairs_host": (_int, [_vp, _vp, _vp, _vp, _sz]),
    "rs_sort_pairs_host_batch": (_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_uint32]),
    "rs_sort_pairs_noalloc": (_int, [_vp, _vp, _sz, _vp]),
    "rs_launch_count": (ctypes.c_uint64, []),
    "rs_profile_enable": (_int, [_int]),
    "rs_profile_read": (_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double), _int]),
    "rs_kernel_kind_name": (ctypes.c_char_p, [_int]),
    "rs_tune_set": (_int, [_int, _int]),
    "rs_tune_get": (_int, [_int]),
    "rs_tune_set_class": (_int, [_int, _int, _int]),
    "rs_tune_get_class": (_int, [_int, _int]),
    "rs_size_class": (_int, [_sz]),
    "rs_graph_create": (_int, [ctypes.POINTER(_vp), _vp, _vp, _sz, _vp, _u32, _vp, _sz]),
    "rs_graph_launch": (_int, [_vp, _vp]),
    "rs_graph_destroy": (_int, [_vp]),
    "rs_tile_shape_count": (_int, []),
    "rs_tile_shape": (_int, [_int, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "rs_debug_set_spin_limit": (_int, [_u32]),
    "rs_debug_withhold_first_tile": (_int, [_int]),
}


class RsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(code, code), status_string(code)))


def lib():
    """The loaded librs.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("librs.so not built: run `python -c \"import __graft_entry__ as g; "
                                  "g.build()\"` or `python -m paper_1008_2849_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().rs_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != RS_OK:
        raise RsError(code, where)


def _dev_ptr(t, name: str, width: int = 4) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.element_size() != width or t.dtype.is_floating_point:
        raise TypeError("%s must hold %d-byte integers, got %s" % (name, width, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def workspace_bytes(n: int, with_values: bool, num_segments: int = 0) -> int:
    return int(lib().rs_workspace_bytes(int(n), 1 if with_values else 0, int(num_segments)))


def alloc_workspace(n: int, with_values: bool, num_segments: int = 0, device=None):
    """A torch uint8 CUDA tensor large enough for an _ex call (256-byte aligned)."""
    import torch
    nbytes = max(workspace_bytes(n, with_values, num_segments), 1)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
    pad = (-ws.data_ptr()) % 256
    return ws[pad:pad + nbytes]


def sort_keys(keys) -> None:
    """Sort a CUDA tensor of keys in place (synchronous)."""
    _check(lib().rs_sort_keys(_dev_ptr(keys, "keys"), keys.numel()), "rs_sort_keys")


def sort_pairs(keys, vals) -> None:
    """Sort (key, value) pairs in place by key, stable (synchronous)."""
    if vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    _check(lib().rs_sort_pairs(_dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), keys.numel()),
           "rs_sort_pairs")


def sort_keys_ex(keys, workspace, stream=None) -> None:
    """Enqueue an in-place keys sort on ``stream`` (default: current stream)."""
    _check(lib().rs_sort_keys_ex(_dev_ptr(keys, "keys"), keys.numel(), _stream_handle(stream),
                                 workspace.data_ptr(), workspace.numel()), "rs_sort_keys_ex")


def sort_pairs_ex(keys, vals, workspace, stream=None) -> None:
    """Enqueue an in-place pairs sort on ``stream`` (default: current stream)."""
    if vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    _check(lib().rs_sort_pairs_ex(_dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), keys.numel(),
                                  _stream_handle(stream), workspace.data_ptr(), workspace.numel()),
           "rs_sort_pairs_ex")


def workspace_bytes_digits11(n: int, with_values: bool) -> int:
    return int(lib().rs_workspace_bytes_digits11(int(n), 1 if with_values else 0))


def alloc_workspace_digits11(n: int, with_values: bool, device=None):
    """A 256-byte aligned torch uint8 CUDA tensor for sort_digits11_ex."""
    import torch
    nbytes = max(workspace_bytes_digits11(n, with_values), 1)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
    pad = (-ws.data_ptr()) % 256
    return ws[pad:pad + nbytes]


def sort_digits11_ex(keys, vals, workspace, stream=None) -> None:
    """Enqueue the in-place sort with three passes of 11/11/10-bit digits
    (vals None: keys only) on ``stream``."""
    if vals is not None and vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    vp = None if vals is None else _dev_ptr(vals, "vals")
    _check(lib().rs_sort_digits11_ex(_dev_ptr(keys, "keys"), vp, keys.numel(),
                                     _stream_handle(stream), workspace.data_ptr(),
                                     workspace.numel()), "rs_sort_digits11_ex")


def _segments(offsets):
    n_seg = offsets.numel() - 1
    if n_seg < 0:
        raise ValueError("offsets must hold num_segments + 1 entries")
    return _dev_ptr(offsets, "offsets"), n_seg


def sort_keys_segmented(keys, offsets) -> None:
    """Sort every segment [offsets[s], offsets[s+1]) of a CUDA key tensor in place."""
    op, ns = _segments(offsets)
    _check(lib().rs_sort_keys_segmented(_dev_ptr(keys, "keys"), keys.numel(), op, ns),
           "rs_sort_keys_segmented")


def sort_pairs_segmented(keys, vals, offsets) -> None:
    """Stable sort of every segment of (key, value) pairs, in place."""
    if vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    op, ns = _segments(offsets)
    _check(lib().rs_sort_pairs_segmented(_dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"),
                                         keys.numel(), op, ns), "rs_sort_pairs_segmented")


def sort_keys_segmented_ex(keys, offsets, workspace, stream=None) -> None:
    op, ns = _segments(offsets)
    _check(lib().rs_sort_keys_segmented_ex(_dev_ptr(keys, "keys"), keys.numel(), op, ns,
                                           _stream_handle(stream), workspace.data_ptr(),
                                           workspace.numel()), "rs_sort_keys_segmented_ex")


def sort_pairs_segmented_ex(keys, vals, offsets, workspace, stream=None) -> None:
    if vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    op, ns = _segments(offsets)
    _check(lib().rs_sort_pairs_segmented_ex(_dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"),
                                            keys.numel(), op, ns, _stream_handle(stream),
                                            workspace.data_ptr(), workspace.numel()),
           "rs_sort_pairs_segmented_ex")


def workspace_bytes64(n: int, with_values: bool) -> int:
    return int(lib().rs_workspace_bytes64(n, 1 if with_values else 0))


def sort64_ex(keys, vals, workspace, stream=None) -> None:
    """Enqueue an in-place sort of 64-bit keys (an int64 CUDA tensor holding
    the uint64 bit patterns), with int32 values or None."""
    if vals is not None and vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    _check(lib().rs_sort64_ex(_dev_ptr(keys, "keys", 8),
                              None if vals is None else _dev_ptr(vals, "vals"), keys.numel(),
                              _stream_handle(stream), workspace.data_ptr(), workspace.numel()),
           "rs_sort64_ex")


# Key types of rs_sort_kv_ex (rs_key_type) and their word widths in bytes.
KV_KEY_TYPES = {"u32": (0, 4), "i32": (1, 4), "f32": (2, 4),
                "u64": (3, 8), "i64": (4, 8), "f64": (5, 8)}


def workspace_bytes_kv(n: int, key_type: str, value_bits: int) -> int:
    return int(lib().rs_workspace_bytes_kv(int(n), KV_KEY_TYPES[key_type][0], int(value_bits)))


def sort_kv_ex(keys, vals, key_type: str, workspace, stream=None) -> None:
    """Enqueue an in-place stable sort of keys read as ``key_type`` (int32
    tensors for the 32-bit types, int64 for the 64-bit ones, holding the bit
    patterns), carrying int32 or int64 values, or None."""
    code, kw = KV_KEY_TYPES[key_type]
    value_bits = 0
    vp = None
    if vals is not None:
        if vals.numel() != keys.numel():
            raise ValueError("keys and vals differ in length")
        value_bits = 8 * vals.element_size()
        vp = _dev_ptr(vals, "vals", vals.element_size())
    _check(lib().rs_sort_kv_ex(_dev_ptr(keys, "keys", kw), vp, keys.numel(), code, value_bits,
                               _stream_handle(stream), workspace.data_ptr(), workspace.numel()),
           "rs_sort_kv_ex")


def sort_kv(keys, vals=None, key_type: str = "u64", stream=None) -> None:
    """Synchronous ``sort_kv_ex`` with a workspace allocated for the call."""
    import torch
    value_bits = 0 if vals is None else 8 * vals.element_size()
    nbytes = max(workspace_bytes_kv(keys.numel(), key_type, value_bits), 1)
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=keys.device)
    pad = (-raw.data_ptr()) % 256
    sort_kv_ex(keys, vals, key_type, raw[pad:pad + nbytes], stream)
    check_stream(stream)


def workspace_bytes_kv_segmented(n: int, key_type: str, value_bits: int, num_segments: int) -> int:
    return int(lib().rs_workspace_bytes_kv_segmented(int(n), KV_KEY_TYPES[key_type][0],
                                                     int(value_bits), int(num_segments)))


def sort_kv_segmented_ex(keys, vals, offsets, key_type: str, workspace, stream=None) -> None:
    """Enqueue the stable sort of every segment [offsets[s], offsets[s+1]) of
    keys read as ``key_type`` (int32 or int64 tensors of bit patterns),
    carrying int32 or int64 values, or None; offsets is an int32 tensor of
    num_segments + 1 entries."""
    code, kw = KV_KEY_TYPES[key_type]
    value_bits = 0
    vp = None
    if vals is not None:
        if vals.numel() != keys.numel():
            raise ValueError("keys and vals differ in length")
        value_bits = 8 * vals.element_size()
        vp = _dev_ptr(vals, "vals", vals.element_size())
    op, ns = _segments(offsets)
    _check(lib().rs_sort_kv_segmented_ex(_dev_ptr(keys, "keys", kw), vp, keys.numel(), op, ns,
                                         code, value_bits, _stream_handle(stream),
                                         workspace.data_ptr(), workspace.numel()),
           "rs_sort_kv_segmented_ex")


def sort_kv_segmented(keys, vals, offsets, key_type: str = "u64", stream=None) -> None:
    """Synchronous ``sort_kv_segmented_ex`` with a workspace allocated for the call."""
    import torch
    value_bits = 0 if vals is None else 8 * vals.element_size()
    nbytes = max(workspace_bytes_kv_segmented(keys.numel(), key_type, value_bits,
                                              offsets.numel() - 1), 1)
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=keys.device)
    pad = (-raw.data_ptr()) % 256
    sort_kv_segmented_ex(keys, vals, offsets, key_type, raw[pad:pad + nbytes], stream)
    check_stream(stream)


def sort64(keys, vals=None, stream=None) -> None:
    """Synchronous 64-bit key sort with a workspace allocated for the call."""
    import torch
    nbytes = max(workspace_bytes64(keys.numel(), vals is not None), 1)
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=keys.device)
    pad = (-raw.data_ptr()) % 256
    sort64_ex(keys, vals, raw[pad:pad + nbytes], stream)
    check_stream(stream)


KEY_TYPES = {"u32": 0, "i32": 1, "f32": 2}


def sort_typed_ex(keys, vals, key_type: str, workspace, stream=None) -> None:
    """Enqueue an in-place sort of keys read as ``key_type`` ("u32", "i32" or
    "f32"; the tensor holds the 32-bit patterns), values optional."""
    if vals is not None and vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    _check(lib().rs_sort_typed_ex(_dev_ptr(keys, "keys"),
                                  None if vals is None else _dev_ptr(vals, "vals"), keys.numel(),
                                  KEY_TYPES[key_type], _stream_handle(stream),
                                  workspace.data_ptr(), workspace.numel()), "rs_sort_typed_ex")


def sort_segmented_typed_ex(keys, vals, offsets, key_type: str, workspace, stream=None) -> None:
    """Enqueue the typed sort of every segment [offsets[s], offsets[s+1])."""
    if vals is not None and vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    op, ns = _segments(offsets)
    _check(lib().rs_sort_segmented_typed_ex(_dev_ptr(keys, "keys"),
                                            None if vals is None else _dev_ptr(vals, "vals"),
                                            keys.numel(), op, ns, KEY_TYPES[key_type],
                                            _stream_handle(stream), workspace.data_ptr(),
                                            workspace.numel()), "rs_sort_segmented_typed_ex")


def sort_typed(keys, vals=None, key_type: str = "f32", offsets=None, stream=None) -> None:
    """Synchronous typed sort (whole array, or per segment with ``offsets``)
    with a workspace allocated for the call; raises on any device error."""
    nseg = 0 if offsets is None else max(offsets.numel() - 1, 0)
    ws = alloc_workspace(keys.numel(), vals is not None, nseg, device=keys.device)
    if offsets is None:
        sort_typed_ex(keys, vals, key_type, ws, stream)
    else:
        sort_segmented_typed_ex(keys, vals, offsets, key_type, ws, stream)
    check_stream(stream)


def stream_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status code."""
    return int(lib().rs_stream_status(_stream_handle(stream)))


def check_stream(stream=None) -> None:
    _check(stream_status(stream), "rs_stream_status")


def msd_partition_ex(keys, vals, out_keys, out_vals, bucket_offsets, workspace,
                     stream=None) -> None:
    """Enqueue Alg. 2's local MSD pass: (keys, vals) stably partitioned by
    their top byte into (out_keys, out_vals); bucket_offsets (257 entries)
    receives every bucket's first slot.  vals and out_vals may both be None."""
    n = keys.numel()
    if out_keys.numel() != n or (vals is not None and (vals.numel() != n or out_vals.numel() != n)):
        raise ValueError("keys, values and outputs differ in length")
    if bucket_offsets.numel() != 257:
        raise ValueError("bucket_offsets must hold 257 entries")
    _check(lib().rs_msd_partition_ex(
        _dev_ptr(keys, "keys"), None if vals is None else _dev_ptr(vals, "vals"), n,
        _dev_ptr(out_keys, "out_keys"), None if out_vals is None else _dev_ptr(out_vals, "out_vals"),
        _dev_ptr(bucket_offsets, "bucket_offsets"), _stream_handle(stream), workspace.data_ptr(),
        workspace.numel()), "rs_msd_partition_ex")


def digit_histograms(keys, out=None, stream=None):
    """(4, 256) int32 CUDA tensor H[p, b] = #keys whose byte p is b."""
    import torch
    if out is None:
        out = torch.empty((4, 256), dtype=torch.int32, device=keys.device)
    _check(lib().rs_digit_histograms_ex(_dev_ptr(keys, "keys"), keys.numel(), _dev_ptr(out, "out"),
                                        _stream_handle(stream)), "rs_digit_histograms_ex")
    return out


def _host_ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or a.element_size() != 4 or not a.is_contiguous():
            raise ValueError("host tensors must be contiguous CPU tensors of 4-byte ints")
        return a.data_ptr()
    if a.dtype.itemsize != 4 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be contiguous 4-byte ints")
    return a.ctypes.data


def _host_len(a) -> int:
    return a.numel() if hasattr(a, "numel") else a.size


def sort_pairs_host(keys_in, vals_in, keys_out, vals_out) -> None:
    """End-to-end sort of host arrays (numpy or CPU torch; pinned is fastest)."""
    _check(lib().rs_sort_pairs_host(_host_ptr(keys_in), _host_ptr(vals_in), _host_ptr(keys_out),
                                    _host_ptr(vals_out), _host_len(keys_in)),
           "rs_sort_pairs_host")


def sort_pairs_host_batch(keys_in, vals_in, keys_out, vals_out) -> None:
    """Pipelined end-to-end sorts of several host arrays (lists of equal
    length; vals_in / vals_out None for keys only): the next array's upload
    and the previous one's download overlap the current sort."""
    count = len(keys_in)
    if len(keys_out) != count or (vals_in is not None and
                                  (len(vals_in) != count or len(vals_out) != count)):
        raise ValueError("input and output lists differ in length")
    P = ctypes.c_void_p * max(count, 1)
    ki = P(*[_host_ptr(a) for a in keys_in])
    ko = P(*[_host_ptr(a) for a in keys_out])
    vi = None if vals_in is None else P(*[_host_ptr(a) for a in vals_in])
    vo = None if vals_out is None else P(*[_host_ptr(a) for a in vals_out])
    n = (ctypes.c_size_t * max(count, 1))(*[_host_len(a) for a in keys_in])
    _check(lib().rs_sort_pairs_host_batch(ki, vi, ko, vo, n, count), "rs_sort_pairs_host_batch")


NOALLOC_MAX_ITEMS = 1 << 20


def sort_pairs_noalloc(keys, vals=None, stream=None) -> None:
    """Enqueue an in-place sort that allocates no device memory (n <= 2^20).

    For callers that must not allocate at call time.  Uses a fixed scratch
    array inside librs.so shared by all calls on a device: calls that overlap
    on the GPU race.  Asynchronous; collect errors with stream_status()."""
    if vals is not None and vals.numel() != keys.numel():
        raise ValueError("keys and vals differ in length")
    _check(lib().rs_sort_pairs_noalloc(_dev_ptr(keys, "keys"),
                                       None if vals is None else _dev_ptr(vals, "vals"),
                                       keys.numel(), _stream_handle(stream)),
           "rs_sort_pairs_noalloc")


def launch_count() -> int:
    return int(lib().rs_launch_count())


def profile_enable(on: bool) -> None:
    _check(lib().rs_profile_enable(1 if on else 0), "rs_profile_enable")


def profile_read() -> dict:
    """{kernel kind: (launches, total_ms)} since the last read; resets tallies."""
    launches = (ctypes.c_uint64 * 16)()
    ms = (ctypes.c_double * 16)()
    k = lib().rs_profile_read(launches, ms, 16)
    out = {}
    for i in range(k):
        name = lib().rs_kernel_kind_name(i).decode()
        out[name] = (int(launches[i]), float(ms[i]))
    return out


TUNE_KNOBS = {"tile_pairs": 0, "tile_keys": 1, "hist_ctas_per_sm": 2, "hist_mode": 3,
              "small_max": 4, "tile_seg": 5, "warp_max": 6, "small_bits": 7, "msd": 8,
              "typed_split": 9, "d11_shape": 10, "digits": 11, "pdl": 13}


def tune_set(knob: str, value: int) -> None:
    _check(lib().rs_tune_set(TUNE_KNOBS[knob], int(value)), "rs_tune_set(%s)" % knob)


def tune_get(knob: str) -> int:
    return int(lib().rs_tune_get(TUNE_KNOBS[knob]))


NUM_SIZE_CLASSES = 6


def tune_set_class(size_class: int, knob: str, value: int) -> None:
    _check(lib().rs_tune_set_class(int(size_class), TUNE_KNOBS[knob], int(value)),
           "rs_tune_set_class(%d, %s)" % (size_class, knob))


def tune_get_class(size_class: int, knob: str) -> int:
    return int(lib().rs_tune_get_class(int(size_class), TUNE_KNOBS[knob]))


def size_class(items: int) -> int:
    return int(lib().rs_size_class(int(items)))


class Graph:
    """A sort of fixed CUDA buffers captured once (rs_graph_create) and
    replayed with one launch per call (rs_graph_launch)."""

    def __init__(self, keys, vals=None, offsets=None, workspace=None):
        n = keys.numel()
        nseg = 0 if offsets is None else offsets.numel() - 1
        if workspace is None:
            workspace = alloc_workspace(n, vals is not None, nseg, device=keys.device)
        self._keep = (keys, vals, offsets, workspace)  # the graph reads these buffers
        h = _vp()
        _check(lib().rs_graph_create(ctypes.byref(h), _dev_ptr(keys, "keys"),
                                     None if vals is None else _dev_ptr(vals, "vals"), n,
                                     None if offsets is None else _dev_ptr(offsets, "offsets"),
                                     nseg, workspace.data_ptr(), workspace.numel()),
               "rs_graph_create")
        self._h = h

    def launch(self, stream=None) -> None:
        _check(lib().rs_graph_launch(self._h, _stream_handle(stream)), "rs_graph_launch")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().rs_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tile_shapes():
    """[(threads, items_per_thread)] of the compiled scatter-pass tile shapes."""
    out = []
    for i in range(int(lib().rs_tile_shape_count())):
        t, j = _int(0), _int(0)
        _check(lib().rs_tile_shape(i, ctypes.byref(t), ctypes.byref(j)), "rs_tile_shape")
        out.append((t.value, j.value))
    return out


def debug_set_spin_limit(iterations: int) -> None:
    _check(lib().rs_debug_set_spin_limit(int(iterations)), "rs_debug_set_spin_limit")


def debug_withhold_first_tile(on: bool) -> None:
    _check(lib().rs_debug_withhold_first_tile(1 if on else 0), "rs_debug_withhold_first_tile")
