"""GPU test of rs_sort_pairs_noalloc, the sort entry point that allocates
nothing (for callers that must not allocate device memory when they sort).

It is called through the C ABI and its output is compared with that of
rs_sort_pairs on the same input, on two calls in a row with different inputs
(the scratch array inside the library keeps the first call's contents, which
must not leak into the second).  Results are integers, so the comparison is
bit-exact.  This file sorts last in collection order on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

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


def test_noalloc_matches_plain_sort_on_two_calls(lib):
    from paper_1008_2849_gb300 import rs
    cases = [("uniform", 1_000_003, 81), ("and2", (1 << 20), 82)]  # second call: the maximum n
    for dist, n, seed in cases:
        k = inputs.keys(dist, n, seed=seed)
        v = inputs.splitmix32(seed, n, 5)
        kd, vd = to_dev(k), to_dev(v)
        _noalloc(lib, kd, vd, n)
        ref_k, ref_v = to_dev(k), to_dev(v)
        rs.sort_pairs(ref_k, ref_v)
        assert np.array_equal(to_host(kd), to_host(ref_k)), (dist, n)
        assert np.array_equal(to_host(vd), to_host(ref_v)), (dist, n)


def test_noalloc_keys_only_and_limits(lib):
    from paper_1008_2849_gb300 import rs
    n = 70_001
    k = inputs.keys("low16", n, seed=83)
    kd = to_dev(k)
    _noalloc(lib, kd, None, n)
    ref = to_dev(k)
    rs.sort_keys(ref)
    assert np.array_equal(to_host(kd), to_host(ref))
    # Beyond the stated maximum the call refuses before touching memory.
    big = to_dev(np.zeros(8, dtype=np.uint32))
    assert lib.rs_sort_pairs_noalloc(big.data_ptr(), None, (1 << 20) + 1, None) == 5
    assert lib.rs_sort_pairs_noalloc(big.data_ptr(), None, 0, None) == 0
