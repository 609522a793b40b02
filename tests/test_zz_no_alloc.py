"""GPU test of rs_sort_pairs_noalloc, the sort entry point that allocates
nothing (for callers that must not allocate device memory when they sort:
latency-critical code, where cudaMalloc and cudaFree can stall the whole
device, and processes whose device memory all belongs to their own pool).

It is called through the C ABI and its output is compared bit for bit with
the CPU oracle's stable sort of the same input (results are integers, so the
comparison is exact).  The cases run as calls in a row with different inputs
and sizes, so the scratch array inside the library holds the previous call's
contents each time; they cover every order the sort takes below the entry
point's maximum: one CTA (n <= 8192), the MSD-first order (n <= 2^16), and
the scatter passes, up to the maximum n.  Each result is also compared with
rs_sort_pairs (the allocating entry point) on the same input.  This file
sorts last in collection order on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs
    build.build_library()
    L = rs.lib()
    L.rs_sort_pairs_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p]
    L.rs_sort_pairs_noalloc.restype = ctypes.c_int
    return L


def _noalloc(lib, kd, vd, n):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.rs_sort_pairs_noalloc(kd.data_ptr(), None if vd is None else vd.data_ptr(), n, stream)
    assert rc == 0, rc
    assert lib.rs_stream_status(stream) == 0


# (distribution, n, seed, with values): calls in this order, in one process.
CASES = [
    ("uniform", 1_000_003, 81, True),    # scatter passes
    ("and2", 1 << 20, 82, True),         # the maximum n
    ("uniform", 50_000, 84, True),       # MSD-first order (n <= 2^16)
    ("low16", 5_000, 85, False),         # one CTA, keys only
    ("uniform", 5_000, 86, True),        # one CTA, pairs
    ("and3", 60_001, 87, False),         # MSD-first order, keys only
    ("uniform", 1 << 20, 88, True),      # the maximum n again, after the small ones
]


def test_noalloc_matches_oracle_on_calls_in_a_row(lib):
    from paper_1008_2849_gb300 import rs
    for dist, n, seed, pairs in CASES:
        k = inputs.keys(dist, n, seed=seed)
        v = inputs.splitmix32(seed, n, 5) if pairs else None
        kd = to_dev(k)
        vd = to_dev(v) if pairs else None
        _noalloc(lib, kd, vd, n)
        ko, vo = oracle.sort_pairs(k, v)
        assert np.array_equal(to_host(kd), ko), (dist, n)
        if pairs:
            assert np.array_equal(to_host(vd), vo), (dist, n)
        # The allocating entry point gives the same bits.
        ref_k = to_dev(k)
        ref_v = to_dev(v) if pairs else None
        if pairs:
            rs.sort_pairs(ref_k, ref_v)
            assert np.array_equal(to_host(vd), to_host(ref_v)), (dist, n)
        else:
            rs.sort_keys(ref_k)
        assert np.array_equal(to_host(kd), to_host(ref_k)), (dist, n)


def test_noalloc_limits(lib):
    # Beyond the stated maximum the call refuses before touching memory.
    big = to_dev(np.zeros(8, dtype=np.uint32))
    assert lib.rs_sort_pairs_noalloc(big.data_ptr(), None, (1 << 20) + 1, None) == 5
    assert lib.rs_sort_pairs_noalloc(big.data_ptr(), None, 0, None) == 0
    assert np.array_equal(to_host(big), np.zeros(8, dtype=np.uint32))
