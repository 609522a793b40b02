"""GPU parity tests of the unsegmented sort: the CUDA path through the C ABI
against the CPU oracle, element by element (bit-exact: all data is integer).

Sizes span one partial tile, several tiles and a ragged tail; the full-size
workloads (2^20 keys; 2^28 pairs; 2^27 pairs in seven key distributions) are
compared in full with the launch configuration the benchmark times.
"""
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
    return _rs


EDGE_SIZES = [1, 2, 31, 32, 33, 255, 256, 257, 4095, 4096, 4097, 6143, 6144, 6145, 8191, 8192,
              8193, 65535, 65537, 1_000_003]


@pytest.mark.parametrize("n", EDGE_SIZES)
def test_pairs_edge_sizes(rs, n):
    k = inputs.keys("uniform", n, seed=100 + n % 97)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    rs.sort_pairs(kd, vd)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko)
    assert np.array_equal(to_host(vd), vo)


@pytest.mark.parametrize("n", [1, 33, 4097, 65537, 999_999])
def test_keys_edge_sizes(rs, n):
    k = inputs.keys("and2", n, seed=200 + n % 89)
    kd = to_dev(k)
    rs.sort_keys(kd)
    assert np.array_equal(to_host(kd), oracle.sort_keys(k))


def test_keys_2pow20_uniform_seed1(rs):
    """2^20 uniform keys, seed 1, keys only, four 8-bit LSD passes (the MSD-
    first order off, as the configuration states), and with it on."""
    n = 1 << 20
    k = inputs.keys("uniform", n, seed=1)
    cls = rs.size_class(n)
    old = rs.tune_get_class(cls, "msd")
    try:
        for msd in (0, 1):
            rs.tune_set_class(cls, "msd", msd)
            kd = to_dev(k)
            rs.sort_keys(kd)
            assert np.array_equal(to_host(kd), oracle.sort_keys(k))
    finally:
        rs.tune_set_class(cls, "msd", old)


def test_pairs_2pow28_uniform(rs):
    """2^28 pairs, uniform keys (seed 2), value = index: the benchmark workload,
    through the same _ex call and workspace the benchmark uses."""
    import torch
    n = 1 << 28
    k = inputs.keys("uniform", n, seed=2)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    ws = rs.alloc_workspace(n, True)
    rs.sort_pairs_ex(kd, vd, ws)
    rs.check_stream()
    ko, vo = oracle_sort(k, v)
    got_k = to_host(kd)
    assert np.array_equal(got_k, ko)
    del got_k
    assert np.array_equal(to_host(vd), vo)
    del kd, vd, ws
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dist", ["uniform", "and2", "and3", "and4", "distinct256", "equal",
                                  "sorted", "reverse", "low16"])
def test_pairs_2pow27_distributions(rs, dist):
    """2^27 pairs, value = index, seeds 3.. per distribution; stability is
    visible through the values."""
    import torch
    n = 1 << 27
    seed = 3 + inputs.DISTRIBUTIONS.index(dist)
    k = inputs.keys(dist, n, seed=seed)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    rs.sort_pairs(kd, vd)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko)
    assert np.array_equal(to_host(vd), vo)
    del kd, vd
    torch.cuda.empty_cache()


def test_digit_histograms(rs):
    for dist, n in (("uniform", 1_000_003), ("equal", 50_000), ("and4", 777_777), ("low16", 3)):
        k = inputs.keys(dist, n, seed=31)
        h = rs.digit_histograms(to_dev(k))
        import torch
        torch.cuda.synchronize()
        got = h.cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, oracle.digit_histograms(k)), dist


def test_digit_histograms_unaligned(rs):
    k = inputs.keys("uniform", 100_001, seed=32)
    for off in (1, 2, 3):
        h = rs.digit_histograms(to_dev(k, offset_elems=off))
        got = h.cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, oracle.digit_histograms(k)), off


@pytest.mark.parametrize("off", [1, 3])
def test_unaligned_base(rs, off):
    n = 300_007
    k = inputs.keys("uniform", n, seed=40 + off)
    v = inputs.index_values(n)
    kd, vd = to_dev(k, offset_elems=off), to_dev(v, offset_elems=off + 1)
    rs.sort_pairs(kd, vd)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)


def test_ex_on_side_stream_twice(rs):
    """Asynchronous calls on a non-default stream, reusing one workspace."""
    import torch
    n = 2_000_003
    s = torch.cuda.Stream()
    ws = rs.alloc_workspace(n, True)
    for seed in (50, 51):
        k = inputs.keys("and3", n, seed=seed)
        v = inputs.splitmix32(seed, n, 7)
        kd, vd = to_dev(k), to_dev(v)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            rs.sort_pairs_ex(kd, vd, ws, stream=s)
        assert rs.stream_status(s) == 0
        ko, vo = oracle_sort(k, v)
        assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)


def test_host_buffers_end_to_end(rs):
    import torch
    n = 3_000_017
    k = inputs.keys("uniform", n, seed=60)
    v = inputs.index_values(n)
    kin = torch.from_numpy(k.view(np.int32)).pin_memory()
    vin = torch.from_numpy(v.view(np.int32)).pin_memory()
    kout = torch.empty_like(kin).pin_memory()
    vout = torch.empty_like(vin).pin_memory()
    rs.sort_pairs_host(kin, vin, kout, vout)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(kout.numpy().view(np.uint32), ko)
    assert np.array_equal(vout.numpy().view(np.uint32), vo)
    assert np.array_equal(kin.numpy().view(np.uint32), k)  # input untouched
    # keys only, pageable numpy arrays, output over the input
    kk = k.copy()
    rs.sort_pairs_host(kk, None, kk, None)
    assert np.array_equal(kk, oracle.sort_keys(k))


def test_host_batch_end_to_end(rs):
    """Pipelined host sorts: arrays of different sizes (one empty, several
    taking the device buffer sets in turn), pairs in pinned memory and
    keys only in pageable memory with outputs over the inputs; every array
    equals the oracle's sort of it alone."""
    import torch
    sizes = [1_000_003, 0, 5, 8192, 2_500_001, 70_001, 1, 300_007]
    ks = [inputs.keys("and2" if i % 2 else "uniform", m, seed=80 + i) for i, m in enumerate(sizes)]
    vs = [inputs.index_values(m) for m in sizes]
    kin = [torch.from_numpy(k.view(np.int32)).pin_memory() for k in ks]
    vin = [torch.from_numpy(v.view(np.int32)).pin_memory() for v in vs]
    kout = [torch.empty_like(t).pin_memory() for t in kin]
    vout = [torch.empty_like(t).pin_memory() for t in vin]
    rs.sort_pairs_host_batch(kin, vin, kout, vout)
    for i, m in enumerate(sizes):
        ko, vo = oracle_sort(ks[i], vs[i])
        assert np.array_equal(kout[i].numpy().view(np.uint32), ko), i
        assert np.array_equal(vout[i].numpy().view(np.uint32), vo), i
        assert np.array_equal(kin[i].numpy().view(np.uint32), ks[i])  # inputs untouched
    kk = [k.copy() for k in ks]
    rs.sort_pairs_host_batch(kk, None, kk, None)
    for i in range(len(sizes)):
        assert np.array_equal(kk[i], oracle.sort_keys(ks[i])), i


def test_lookback_wait_runs_out(rs):
    """The first tile withholds its counts, so later tiles' bounded waits run
    out: the call reports RS_ERR_TIMEOUT and the context stays usable."""
    n = 5 * 8192 + 11
    k = inputs.keys("uniform", n, seed=70)
    v = inputs.index_values(n)
    kd, vd = to_dev(k), to_dev(v)
    rs.debug_set_spin_limit(2000)
    rs.debug_withhold_first_tile(True)
    try:
        with pytest.raises(rs.RsError) as ei:
            rs.sort_pairs(kd, vd)
        assert ei.value.code == 4
    finally:
        rs.debug_withhold_first_tile(False)
        rs.debug_set_spin_limit(0)
    # The device is still usable and the status word was cleared.
    assert rs.stream_status() == 0
    kd, vd = to_dev(k), to_dev(v)
    rs.sort_pairs(kd, vd)
    ko, vo = oracle_sort(k, v)
    assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo)


def test_wide_status_2pow30_plus(rs):
    """n >= 2^30 switches the look-back to 64-bit status words.  At this size
    the result is checked through properties that hold at any size, on the
    device: nondecreasing keys, values a permutation, each key travelling
    with its value, and equal keys keeping input order."""
    import torch
    n = (1 << 30) + 4099
    # Keys: a fixed device-side hash of the index (a test input; no oracle
    # value is derived from it).
    idx = torch.arange(n, dtype=torch.int64, device="cuda")
    gen_k = ((idx * 0x9E3779B1) ^ (idx >> 7)) & 0xFFFF_FFF0   # many ties in the low bits
    keys = gen_k.to(torch.int32)                              # bit pattern of the uint32 key
    orig = keys.clone()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    del gen_k, idx
    rs.sort_pairs(keys, vals)
    ku = keys.to(torch.int64) & 0xFFFFFFFF
    assert bool((ku[1:] >= ku[:-1]).all())
    # Range first: indexing by an out-of-range value would be a device-side error.
    assert bool(((vals >= 0) & (vals.long() < n)).all())
    assert bool((orig[vals.long()] == keys).all())
    same = ku[1:] == ku[:-1]
    assert bool((vals[1:][same] > vals[:-1][same]).all())
    assert int(vals.long().sum()) == n * (n - 1) // 2
    seen = torch.zeros(n, dtype=torch.bool, device="cuda")
    seen[vals.long()] = True
    assert bool(seen.all())


def _plan_slots_used(ws):
    """Tiles taken per plan slot by the last sort that used workspace `ws`:
    the control block sits at the start of the workspace (err, then nine
    tile counters: LSD passes 0..7 -- 0..3 for 32-bit keys -- and the MSD
    pass).  Returns [passes 0..3, MSD pass]."""
    head = ws[:40].cpu().numpy().view(np.uint32)
    return head[1:5].tolist() + [int(head[9])]


def _msd_keys(kind, n, seed):
    if kind == "top_few":          # top byte in 0..3: four large buckets
        k = inputs.keys("uniform", n, seed) & np.uint32(0x03FFFFFF)
    elif kind == "lone_bucket":    # plus one key alone in bucket 255 (a size-1 bucket)
        k = inputs.keys("uniform", n, seed) & np.uint32(0x03FFFFFF)
        k[n // 2] = 0xFF000001
    else:
        k = inputs.keys(kind, n, seed)
    return k


@pytest.mark.parametrize("kind,n,taken", [
    ("uniform", 8193, True), ("uniform", 65_537, True), ("uniform", (1 << 18) + 5, True),
    ("uniform", 1 << 20, True), ("uniform", (1 << 21) - 3, None),
    ("top_few", 20_000, True), ("lone_bucket", 9_000, True),
    ("low16", 100_000, False),        # top digit constant: the MSD pass would do nothing
    ("and4", 1 << 20, False),         # top-digit bucket 0 far above 8192 keys
])
def test_msd_first_order(rs, kind, n, taken):
    """Whole arrays that may take the MSD-first order of Alg. 2 (one pass by
    the top digit, then every bucket sorted on chip): the result equals the
    oracle's LSD sort whichever order the plan chose, with the MSD order on
    and off, pairs and keys; where the choice is fixed by the data, the plan
    is checked to have made it."""
    import torch
    k = _msd_keys(kind, n, seed=300 + n % 89)
    v = inputs.index_values(n)
    ko, vo = oracle_sort(k, v)
    cls = rs.size_class(n)
    old = rs.tune_get_class(cls, "msd")
    try:
        for msd in (1, 0):
            rs.tune_set_class(cls, "msd", msd)
            for pairs in (True, False):
                kd, vd = to_dev(k), to_dev(v)
                ws = rs.alloc_workspace(n, pairs)
                if pairs:
                    rs.sort_pairs_ex(kd, vd, ws)
                else:
                    rs.sort_keys_ex(kd, ws)
                rs.check_stream()
                assert np.array_equal(to_host(kd), ko), (kind, n, msd, pairs)
                if pairs:
                    assert np.array_equal(to_host(vd), vo), (kind, n, msd, pairs)
                tiles = _plan_slots_used(ws)
                used_msd = tiles[4] > 0
                if msd == 0 or n > (1 << 21):
                    assert not used_msd
                elif taken is not None:
                    assert used_msd == taken, (kind, n, tiles)
                if used_msd:
                    assert tiles[:4] == [0, 0, 0, 0]
                torch.cuda.synchronize()
    finally:
        rs.tune_set_class(cls, "msd", old)
