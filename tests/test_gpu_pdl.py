"""GPU parity tests of the launch chains with and without programmatic
dependent launch (RS_TUNE_PDL): every kernel of a chain may become resident
while the kernel before it finishes, and must wait on the device before it
reads that kernel's output.

Each case sorts, on one stream and with no host synchronisation in between,
a sequence of different sorts -- a whole array of pairs, a small array (the
one-CTA sort), a segmented batch (planner, one-warp and one-CTA sorts,
segment histograms and scan, scatter passes), float keys, 64-bit keys, and
the same arrays again in place -- so that every chain follows another, and
checks all results against the CPU oracle, bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs
from tests.gpu_util import oracle_sort, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    old = _rs.tune_get("pdl")
    yield _rs
    _rs.tune_set("pdl", old)


def _aligned(torch, nbytes):
    raw = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device="cuda")
    return raw[(-raw.data_ptr()) % 256:][:max(nbytes, 1)]


@pytest.mark.parametrize("pdl", [0, 1])
def test_chains_back_to_back(rs, pdl):
    import torch
    rs.tune_set("pdl", pdl)
    stream = torch.cuda.Stream()
    # 1. whole array of pairs, several tiles and a ragged end.
    n1 = (1 << 20) + 77
    k1 = inputs.keys("and2", n1, seed=800 + pdl)
    v1 = inputs.index_values(n1)
    # 2. a small array: the one-CTA sort.
    n2 = 5_001
    k2 = inputs.keys("uniform", n2, seed=801)
    v2 = inputs.index_values(n2)
    # 3. a segmented batch with one-warp, one-CTA and scatter-pass segments.
    k3, v3, off3 = inputs.segmented_batch(96, 1, 17, seed=802)
    # 4. float keys.
    n4 = 300_001
    k4 = inputs.keys("uniform", n4, seed=803)
    v4 = inputs.index_values(n4)
    # 5. 64-bit keys.
    n5 = 200_003
    hi = inputs.splitmix32(804, n5, 0).astype(np.uint64)
    k5 = (hi << np.uint64(32)) | inputs.splitmix32(804, n5, 1).astype(np.uint64)
    v5 = inputs.index_values(n5)

    d1k, d1v = to_dev(k1), to_dev(v1)
    d2k, d2v = to_dev(k2), to_dev(v2)
    d3k, d3v, d3o = to_dev(k3), to_dev(v3), to_dev(off3)
    d4k, d4v = to_dev(k4), to_dev(v4)
    d5k = torch.from_numpy(k5.view(np.int64)).cuda()
    d5v = to_dev(v5)
    ws1 = rs.alloc_workspace(n1, True)
    ws2 = rs.alloc_workspace(n2, True)
    ws3 = rs.alloc_workspace(k3.size, True, off3.size - 1)
    ws4 = rs.alloc_workspace(n4, True)
    ws5 = _aligned(torch, rs.workspace_bytes64(n5, True))
    torch.cuda.synchronize()
    for _ in range(2):  # the second round sorts sorted data again: same result
        rs.sort_pairs_ex(d1k, d1v, ws1, stream=stream)
        rs.sort_pairs_ex(d2k, d2v, ws2, stream=stream)
        rs.sort_pairs_segmented_ex(d3k, d3v, d3o, ws3, stream=stream)
        rs.sort_typed_ex(d4k, d4v, "f32", ws4, stream=stream)
        rs.sort64_ex(d5k, d5v, ws5, stream=stream)
    rs.check_stream(stream)
    torch.cuda.synchronize()

    ko, vo = oracle_sort(k1, v1)
    assert np.array_equal(to_host(d1k), ko) and np.array_equal(to_host(d1v), vo)
    ko, vo = oracle_sort(k2, v2)
    assert np.array_equal(to_host(d2k), ko) and np.array_equal(to_host(d2v), vo)
    ko, vo = oracle.sort_pairs_segmented(k3, v3, off3)
    assert np.array_equal(to_host(d3k), ko) and np.array_equal(to_host(d3v), vo)
    ko, vo = oracle.sort_typed(k4, v4, "f32")
    assert np.array_equal(to_host(d4k), ko) and np.array_equal(to_host(d4v), vo)
    ko, vo = oracle.sort_pairs64(k5, v5)
    assert np.array_equal(d5k.cpu().numpy().view(np.uint64), ko)
    assert np.array_equal(to_host(d5v), vo)
