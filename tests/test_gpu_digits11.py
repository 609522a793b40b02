"""GPU parity tests of the sort with three passes of 11/11/10-bit digits
(rs_sort_digits11_ex; Sec. 4 with D = 11) against the CPU oracle, bit for bit.

The oracle's stable sort does not depend on the digit width, so the result
must equal oracle.sort_pairs (keys and values) for every size and key
distribution: one item, one partial tile, tile edges, several chunks with
ragged ends, and skewed keys (AND of several draws, 16-bit keys, one value,
256 distinct values).  At 2^28 pairs the whole output is checked by
properties that pin the stable sort at any size: keys nondecreasing, values
a permutation of the input indices, every output key the input key at its
value's index, and equal keys in index order."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1008_2849_gb300 import inputs
from tests.gpu_util import oracle_sort, to_dev, to_host

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 4095, 4096, 4097, 70_001, 1_000_003, (1 << 22) + 11, (1 << 24) + 3]
DISTS = ["uniform", "and3", "low16", "equal", "distinct256"]


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dist_name", DISTS)
def test_digits11_pairs_match_oracle(rs, n, dist_name):
    k = inputs.keys(dist_name, n, seed=600 + n % 97)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    ws = rs.alloc_workspace_digits11(n, True)
    rs.sort_digits11_ex(kd, vd, ws)
    rs.check_stream()
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko)
    assert np.array_equal(to_host(vd), vo)


@pytest.mark.parametrize("n", [1, 4097, 1_000_003, (1 << 24) + 3])
@pytest.mark.parametrize("dist_name", ["uniform", "and2"])
def test_digits11_keys_match_oracle(rs, n, dist_name):
    k = inputs.keys(dist_name, n, seed=610 + n % 89)
    kd = to_dev(k)
    ws = rs.alloc_workspace_digits11(n, False)
    rs.sort_digits11_ex(kd, None, ws)
    rs.check_stream()
    ko, _ = oracle_sort(k, None)
    assert np.array_equal(to_host(kd), ko)


@pytest.mark.parametrize("off_elems", [1, 3])
def test_digits11_unaligned(rs, off_elems):
    """Arrays that start only 4-byte aligned."""
    n = 300_007
    k = inputs.keys("and2", n, seed=620)
    v = inputs.splitmix32(621, n, 1)
    kd, vd = to_dev(k, off_elems), to_dev(v, off_elems)
    ws = rs.alloc_workspace_digits11(n, True)
    rs.sort_digits11_ex(kd, vd, ws)
    rs.check_stream()
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)


def test_digits11_workspace_errors(rs):
    import torch
    kd = to_dev(np.arange(1000, dtype=np.uint32))
    ws = rs.alloc_workspace_digits11(1000, False)
    with pytest.raises(rs.RsError):
        rs.sort_digits11_ex(kd, None, ws[:256])
    with pytest.raises(rs.RsError):  # pairs need the larger workspace
        rs.sort_digits11_ex(kd, torch.empty_like(kd), ws)
    assert rs.stream_status() == 0


def test_digits11_full_size_properties(rs):
    """2^28 pairs (uniform keys, index values): the stable sort checked by
    properties over the whole output, and 4096 sampled positions against
    the rank of their key counted on the host."""
    import torch
    n = 1 << 28
    kd = inputs.keys_torch("uniform", n, seed=630)
    vd = torch.arange(n, dtype=torch.int32, device="cuda")
    k_in = kd.clone()
    ws = rs.alloc_workspace_digits11(n, True)
    rs.sort_digits11_ex(kd, vd, ws)
    rs.check_stream()
    ku = kd.to(torch.int64) & 0xFFFFFFFF
    assert bool((ku[1:] >= ku[:-1]).all())
    vi = vd.to(torch.int64)
    ki = k_in.to(torch.int64) & 0xFFFFFFFF
    assert bool((ki[vi] == ku).all())                  # every key travels with its index
    assert int(torch.bincount(vi, minlength=n).max()) == 1   # a permutation
    eq = ku[1:] == ku[:-1]
    assert bool((vi[1:][eq] > vi[:-1][eq]).all())      # stable
    del ws, k_in
    # Sampled ranks against the host: the key at output position p is the
    # smallest key with more than p keys <= it.
    host = ki.cpu().numpy()
    srt = np.sort(host)
    pos = (inputs.splitmix32(631, 4096, 0).astype(np.int64) * n) >> 32
    assert np.array_equal(ku[torch.from_numpy(pos).cuda()].cpu().numpy(), srt[pos])
