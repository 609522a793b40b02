"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle's.

This module holds no sorting arithmetic: it only draws keys, values, segment
tables and request streams.  The paper draws uniform 32-bit keys with WELL512
(Sec. 5); sorting results do not depend on the generator, so a counter-based
generator with a published definition is used instead: SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
keeping the upper 32 bits of every 64-bit output.

Stream ``k`` of seed ``s`` starts from state ``s * 256 + k``; output ``i``
(0-based) is ``mix(state + (i + 1) * 0x9E3779B97F4A7C15) >> 32`` where ``mix``
is the SplitMix64 finaliser.

Distributions (names used by tests and the benchmark):

* ``uniform``     -- stream 0.
* ``and2/3/4``    -- bitwise AND of streams 0..k-1 (bit-one probability 2^-k).
* ``distinct256`` -- 256 table words from stream 1, index = stream 0 >> 24.
* ``equal``       -- every key equal to word 0 of stream 0.
* ``sorted``      -- the uniform keys in ascending order.
* ``reverse``     -- the uniform keys in descending order.
* ``low16``       -- uniform keys AND 0xFFFF.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 20

DISTRIBUTIONS = ("uniform", "and2", "and3", "and4", "distinct256", "equal",
                 "sorted", "reverse", "low16")


def splitmix32(seed: int, n: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """Upper 32 bits of SplitMix64 outputs ``start .. start+n-1`` of a stream."""
    out = np.empty(n, dtype=np.uint32)
    if n == 0:
        return out
    s0 = np.uint64((seed * 256 + stream) & 0xFFFFFFFFFFFFFFFF)
    chunk = min(_CHUNK, n)
    z = np.empty(chunk, dtype=np.uint64)
    t = np.empty(chunk, dtype=np.uint64)
    ramp = np.arange(1, chunk + 1, dtype=np.uint64)
    s30, s27, s31, s32 = (np.uint64(x) for x in (30, 27, 31, 32))
    with np.errstate(over="ignore"):
        for c in range(0, n, chunk):
            m = min(chunk, n - c)
            zz, tt = z[:m], t[:m]
            np.add(ramp[:m], np.uint64(start + c), out=zz)
            np.multiply(zz, GOLDEN, out=zz)
            np.add(zz, s0, out=zz)
            np.right_shift(zz, s30, out=tt)
            np.bitwise_xor(zz, tt, out=zz)
            np.multiply(zz, _M1, out=zz)
            np.right_shift(zz, s27, out=tt)
            np.bitwise_xor(zz, tt, out=zz)
            np.multiply(zz, _M2, out=zz)
            np.right_shift(zz, s31, out=tt)
            np.bitwise_xor(zz, tt, out=zz)
            np.right_shift(zz, s32, out=tt)
            out[c:c + m] = tt
    return out


def _as_i64(x: int) -> int:
    """The 64-bit two's-complement value of an unsigned 64-bit constant."""
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >= (1 << 63) else x


def splitmix32_torch(seed: int, n: int, stream: int = 0, start: int = 0, device="cuda", out=None):
    """The same words as ``splitmix32``, computed with torch int64 arithmetic
    (wrapping multiplication; right shifts masked to be logical), returned
    as an int32 tensor holding the uint32 bit patterns.  Used to draw large
    serving workloads on the device; a CPU test pins it to ``splitmix32``."""
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=device)
    if n == 0:
        return out
    s0 = _as_i64(seed * 256 + stream)
    g, m1, m2 = _as_i64(0x9E3779B97F4A7C15), _as_i64(0xBF58476D1CE4E5B9), _as_i64(0x94D049BB133111EB)
    chunk = 1 << 26
    for c in range(0, n, chunk):
        m = min(chunk, n - c)
        z = torch.arange(start + c + 1, start + c + m + 1, dtype=torch.int64, device=out.device)
        z.mul_(g).add_(s0)
        z.bitwise_xor_((z >> 30) & ((1 << 34) - 1)).mul_(m1)
        z.bitwise_xor_((z >> 27) & ((1 << 37) - 1)).mul_(m2)
        z.bitwise_xor_((z >> 31) & ((1 << 33) - 1))
        out[c:c + m] = ((z >> 32) & 0xFFFFFFFF).to(torch.int32)
    return out


def keys_torch(dist: str, n: int, seed: int, device="cuda", out=None):
    """Device-side ``keys`` for the distributions the serving workload uses
    (``uniform`` and ``and2``); int32 tensor of uint32 bit patterns."""
    out = splitmix32_torch(seed, n, 0, device=device, out=out)
    if dist == "uniform":
        return out
    if dist == "and2":
        out.bitwise_and_(splitmix32_torch(seed, n, 1, device=out.device))
        return out
    raise ValueError("device-side generator supports uniform and and2, not %r" % dist)


def keys(dist: str, n: int, seed: int) -> np.ndarray:
    """``n`` uint32 keys of distribution ``dist`` (see module docstring)."""
    if dist == "uniform":
        return splitmix32(seed, n, 0)
    if dist in ("and2", "and3", "and4"):
        k = int(dist[3])
        out = splitmix32(seed, n, 0)
        for s in range(1, k):
            np.bitwise_and(out, splitmix32(seed, n, s), out=out)
        return out
    if dist == "distinct256":
        table = splitmix32(seed, 256, 1)
        idx = splitmix32(seed, n, 0) >> np.uint32(24)
        return table[idx]
    if dist == "equal":
        return np.full(n, splitmix32(seed, 1, 0)[0], dtype=np.uint32)
    if dist == "sorted":
        return np.sort(splitmix32(seed, n, 0))
    if dist == "reverse":
        return np.ascontiguousarray(np.sort(splitmix32(seed, n, 0))[::-1])
    if dist == "low16":
        return splitmix32(seed, n, 0) & np.uint32(0xFFFF)
    raise ValueError("unknown distribution %r" % dist)


def index_values(n: int) -> np.ndarray:
    """Values equal to the input index, so stability is visible in the output."""
    return np.arange(n, dtype=np.uint32)


def uniform01(seed: int, n: int, stream: int) -> np.ndarray:
    """Floats in [0, 1) built from the 32-bit words of a stream."""
    return splitmix32(seed, n, stream).astype(np.float64) / 4294967296.0


def loguniform_segment_sizes(num_segments: int, lo_log2: float, hi_log2: float,
                             seed: int) -> np.ndarray:
    """Segment sizes floor(2^U), U uniform on [lo_log2, hi_log2] (uint64)."""
    u = uniform01(seed, num_segments, 0)
    return np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.uint64)


def offsets_from_sizes(sizes) -> np.ndarray:
    """Segment table with len(sizes)+1 entries: 0, then running totals."""
    sizes = np.asarray(sizes, dtype=np.uint64)
    off = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=off[1:])
    if off[-1] >= (1 << 32):
        raise ValueError("segment table total exceeds 32 bits")
    return off.astype(np.uint32)


def segmented_batch(num_segments: int, lo_log2: float, hi_log2: float, seed: int,
                    scale_to: int | None = None):
    """Batch of independent arrays: (keys, values, offsets).

    Sizes are log-uniform; keys are uniform; the value of an item is its index
    inside its own segment.  ``scale_to`` rescales the drawn sizes so that they
    total about that many items (floor, at least 1 each).
    """
    sizes = loguniform_segment_sizes(num_segments, lo_log2, hi_log2, seed)
    if scale_to is not None:
        sizes = np.maximum(np.floor(sizes.astype(np.float64) * (scale_to / float(sizes.sum()))),
                           1).astype(np.uint64)
    off = offsets_from_sizes(sizes)
    n = int(off[-1])
    k = splitmix32(seed, n, 1)
    v = (np.arange(n, dtype=np.uint64) - np.repeat(off[:-1].astype(np.uint64),
                                                   sizes.astype(np.int64))).astype(np.uint32)
    return k, v, off


def request_stream(num_requests: int, seed: int, lo_log10: float = 3.0,
                   hi_log10: float = 8.0, pair_fraction: float = 0.3):
    """Serving workload: per request (size, with_values, dist, key_seed).

    Sizes are floor(10^U), U uniform on [lo_log10, hi_log10]; ``with_values`` is
    true with probability ``pair_fraction``; keys are ``uniform`` or ``and2``
    with equal probability.  Arrival times are drawn separately by
    ``poisson_arrivals`` once the rate is known.
    """
    u_size = uniform01(seed, num_requests, 0)
    u_kind = uniform01(seed, num_requests, 1)
    u_dist = uniform01(seed, num_requests, 2)
    sizes = np.floor(np.power(10.0, lo_log10 + (hi_log10 - lo_log10) * u_size)).astype(np.int64)
    reqs = []
    for i in range(num_requests):
        reqs.append(dict(id=i, n=int(sizes[i]), with_values=bool(u_kind[i] < pair_fraction),
                         dist="uniform" if u_dist[i] < 0.5 else "and2",
                         key_seed=seed * 1000003 + i))
    return reqs


def poisson_arrivals(num_requests: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    u = uniform01(seed, num_requests, 3)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
