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


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [5000, 1_000_003])
def test_digits11_every_tile_shape(rs, shape, n):
    """Every tile shape of the scatter kernel (RS_TUNE_D11_SHAPE), pairs and
    keys only."""
    old = rs.tune_get("d11_shape")
    rs.tune_set("d11_shape", shape)
    try:
        k = inputs.keys("and2", n, seed=640 + shape)
        v = inputs.index_values(n)
        kd, vd, kk = to_dev(k), to_dev(v), to_dev(k)
        rs.sort_digits11_ex(kd, vd, rs.alloc_workspace_digits11(n, True))
        rs.sort_digits11_ex(kk, None, rs.alloc_workspace_digits11(n, False))
        rs.check_stream()
    finally:
        rs.tune_set("d11_shape", old)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)
    assert np.array_equal(to_host(kk), ko)


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


@pytest.mark.parametrize("pairs", [True, False])
def test_digits_knob_routes_the_plain_sorts(rs, pairs):
    """RS_TUNE_DIGITS = 11 in the array's size class: the plain call, the
    _ex call with a workspace from rs_workspace_bytes, and a captured graph
    all run the three 11/11/10-bit passes (their kernels are the ones that
    launch) and equal the oracle; with an 8-bit-sized workspace the _ex call
    takes the 8-bit passes, with the same result."""
    n = 1_000_003
    cls = rs.size_class(n)
    k = inputs.keys("uniform", n, seed=650 + pairs)
    v = inputs.index_values(n)
    ko, vo = oracle_sort(k, v)
    old = rs.tune_get_class(cls, "digits")
    rs.profile_enable(True)
    try:
        small_ws = rs.alloc_workspace(n, pairs)  # sized for the 8-bit order
        rs.tune_set_class(cls, "digits", 11)
        outs = []
        for how in ("plain", "ex", "graph", "ex_small"):
            kd, vd = to_dev(k), to_dev(v)
            rs.profile_read()
            launches = rs.launch_count()
            if how == "plain":
                rs.sort_pairs(kd, vd) if pairs else rs.sort_keys(kd)
            elif how in ("ex", "ex_small"):
                ws = small_ws if how == "ex_small" else rs.alloc_workspace(n, pairs)
                rs.sort_pairs_ex(kd, vd, ws) if pairs else rs.sort_keys_ex(kd, ws)
            else:
                g = rs.Graph(kd, vd if pairs else None)
                g.launch()
                g.close()
            rs.check_stream()
            prof = rs.profile_read()
            launched = rs.launch_count() - launches
            if how == "graph":  # replays are counted, not timed per kernel
                assert launched == 9, launched  # 3 x (count, scan, scatter)
            elif how == "ex_small":
                assert "d11_down" not in prof or prof["d11_down"][0] == 0, prof
            else:
                assert prof["d11_down"][0] == 3 and launched == 9, (how, prof, launched)
            outs.append((how, to_host(kd), to_host(vd)))
    finally:
        rs.profile_enable(False)
        rs.tune_set_class(cls, "digits", old)
    for how, ok_, ov_ in outs:
        assert np.array_equal(ok_, ko), how
        if pairs:
            assert np.array_equal(ov_, vo), how
