"""GPU parity tests of the segmented sort (and of the one-warp and one-CTA
sorts it uses for tiny and small segments) against the CPU oracle, element by
element.

The segmented sort has no counterpart in the paper: it is the paper's sort
applied to every segment [off[s], off[s+1]) on its own, which is exactly what
oracle.sort_pairs_segmented computes.
"""
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


def _check_segmented(rs, k, v, off, keys_only=False):
    kd = to_dev(k)
    od = to_dev(off)
    if keys_only:
        rs.sort_keys_segmented(kd, od)
        ko, _ = oracle.sort_pairs_segmented(k, None, off)
        assert np.array_equal(to_host(kd), ko)
        return
    vd = to_dev(v)
    rs.sort_pairs_segmented(kd, vd, od)
    ko, vo = oracle.sort_pairs_segmented(k, v, off)
    assert np.array_equal(to_host(kd), ko)
    assert np.array_equal(to_host(vd), vo)


EDGE_SIZES = [0, 1, 2, 3, 5, 31, 32, 33, 255, 256, 257, 4095, 4096, 4097, 8191, 8192, 8193,
              9000, 100_000, 0, 1, 70_001, 4608, 4609, 2]


@pytest.mark.parametrize("keys_only", [False, True])
def test_segment_edge_sizes(rs, keys_only):
    sizes = np.array(EDGE_SIZES, dtype=np.uint64)
    lead, tail = 7, 11  # items before the first and after the last segment stay put
    off = (inputs.offsets_from_sizes(sizes).astype(np.uint64) + lead).astype(np.uint32)
    n = int(off[-1]) + tail
    k = inputs.keys("and2", n, seed=90)
    v = inputs.index_values(n)
    _check_segmented(rs, k, v, off, keys_only)


@pytest.mark.parametrize("small_max", [4096, 8192])
@pytest.mark.parametrize("tile_seg", [0, 3])
def test_segmented_batch_knobs(rs, small_max, tile_seg):
    """512 arrays, sizes log-uniform on [2^8, 2^17], uniform keys, value =
    index inside the segment; the result may not depend on the tuning."""
    k, v, off = inputs.segmented_batch(512, 8, 17, seed=91)
    old = (rs.tune_get("small_max"), rs.tune_get("tile_seg"))
    rs.tune_set("small_max", small_max)
    rs.tune_set("tile_seg", tile_seg)
    try:
        _check_segmented(rs, k, v, off)
    finally:
        rs.tune_set("small_max", old[0])
        rs.tune_set("tile_seg", old[1])


def test_segmented_4096_arrays_scaled_to_2pow28(rs):
    """4096 arrays with sizes log-uniform on [2^8, 2^22] (seed 10), rescaled
    so that they total about 2^28 pairs; uniform keys, value = index inside
    the segment; through the _ex call on the current stream."""
    import torch
    k, v, off = inputs.segmented_batch(4096, 8, 22, seed=10, scale_to=1 << 28)
    n = k.size
    kd, vd, od = to_dev(k), to_dev(v), to_dev(off)
    ws = rs.alloc_workspace(n, True, num_segments=off.size - 1)
    rs.sort_pairs_segmented_ex(kd, vd, od, ws)
    rs.check_stream()
    ko, vo = oracle.sort_pairs_segmented(k, v, off)
    assert np.array_equal(to_host(kd), ko)
    assert np.array_equal(to_host(vd), vo)
    del kd, vd, od, ws
    torch.cuda.empty_cache()


def test_segmented_4096_arrays_full_size_properties(rs):
    """4096 arrays with sizes log-uniform on [2^8, 2^22] (seed 10), about
    1.77e9 pairs in total.  At this size the result is checked on the device
    through properties that hold at any size: inside every segment keys are
    nondecreasing and equal keys keep their values (= index inside the
    segment) increasing; values are a permutation of 0..size-1 per segment
    (their sum and their bitwise XOR match), and every key moved with its
    value (sum of keys per segment is unchanged)."""
    import torch
    sizes = inputs.loguniform_segment_sizes(4096, 8, 22, seed=10)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    # Keys are drawn on the host in chunks to bound host memory.
    kd = torch.empty(n, dtype=torch.int32, device="cuda")
    chunk = 1 << 27
    for c in range(0, n, chunk):
        m = min(chunk, n - c)
        kd[c:c + m] = torch.from_numpy(inputs.splitmix32(10, m, 1, start=c).view(np.int32)).cuda()
    od = torch.from_numpy(off.view(np.int32)).cuda()
    seg_id = torch.repeat_interleave(torch.arange(4096, device="cuda"),
                                     torch.from_numpy(sizes.astype(np.int64)).cuda())
    starts = od[:-1].long() & 0xFFFFFFFF
    vd = (torch.arange(n, device="cuda", dtype=torch.int64) - starts[seg_id]).to(torch.int32)
    key_sum_before = torch.zeros(4096, dtype=torch.int64, device="cuda").index_add_(
        0, seg_id, kd.long() & 0xFFFFFFFF)
    rs.sort_pairs_segmented(kd, vd, od)
    ku = kd.long() & 0xFFFFFFFF
    same_seg = seg_id[1:] == seg_id[:-1]
    assert bool(((ku[1:] >= ku[:-1]) | ~same_seg).all())
    eq = same_seg & (ku[1:] == ku[:-1])
    assert bool((vd[1:][eq] > vd[:-1][eq]).all())
    sz = torch.from_numpy(sizes.astype(np.int64)).cuda()
    vsum = torch.zeros(4096, dtype=torch.int64, device="cuda").index_add_(0, seg_id, vd.long())
    assert bool((vsum == sz * (sz - 1) // 2).all())
    key_sum_after = torch.zeros(4096, dtype=torch.int64, device="cuda").index_add_(0, seg_id, ku)
    assert bool((key_sum_after == key_sum_before).all())
    assert int(vd.min()) == 0 and bool((vd.long() < sz[seg_id]).all())


def test_bad_segment_table_writes_nothing(rs):
    n = 10_000
    k = inputs.keys("uniform", n, seed=92)
    v = inputs.index_values(n)
    for off in (np.array([0, 5000, 4000, 10_000], dtype=np.uint32),     # decreasing
                np.array([0, 5000, 10_001], dtype=np.uint32)):          # past n
        kd, vd = to_dev(k), to_dev(v)
        with pytest.raises(rs.RsError) as ei:
            rs.sort_pairs_segmented(kd, vd, to_dev(off))
        assert ei.value.code == 7
        assert np.array_equal(to_host(kd), k) and np.array_equal(to_host(vd), v)
    assert rs.stream_status() == 0


def test_one_cta_sort_sizes(rs):
    """Whole arrays small enough for the one-CTA shared-memory sort."""
    old = rs.tune_get("small_max")
    rs.tune_set("small_max", 8192)
    try:
        for n, dist in ((2, "uniform"), (100, "equal"), (4096, "and4"), (5000, "low16"),
                        (8192, "uniform"), (8191, "distinct256")):
            k = inputs.keys(dist, n, seed=93)
            v = inputs.index_values(n)
            kd, vd = to_dev(k), to_dev(v)
            rs.sort_pairs(kd, vd)
            ko, vo = oracle.sort_pairs(k, v)
            assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo), (n, dist)
    finally:
        rs.tune_set("small_max", old)


def _with_knobs(rs, settings, fn):
    """Run fn() with per-class knobs set in every class, then restore them."""
    saved = [(c, k, rs.tune_get_class(c, k)) for c in range(6) for k in settings]
    try:
        for k, v in settings.items():
            rs.tune_set(k, v)
        fn()
    finally:
        for c, k, v in saved:
            rs.tune_set_class(c, k, v)


TINY_SIZES = [0, 1, 2, 3, 17, 31, 32, 33, 63, 64, 65, 100, 255, 256, 257, 300, 511, 512, 513,
              600, 1000, 4096, 4097, 5000, 1, 2, 480]


@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("warp_max", [0, 256, 512])
def test_tiny_segments_warp_sort(rs, bits, warp_max):
    """Segments around the one-warp sort's capacity, at both digit widths and
    with the one-warp sort off, at 256 and at 512 items."""
    sizes = np.array(TINY_SIZES * 3, dtype=np.uint64)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    for dist in ("uniform", "and4", "low16", "equal"):
        k = inputs.keys(dist, n, seed=94)
        v = inputs.index_values(n)
        _with_knobs(rs, {"warp_max": warp_max, "small_bits": bits},
                    lambda: _check_segmented(rs, k, v, off))
        _with_knobs(rs, {"warp_max": warp_max, "small_bits": bits},
                    lambda: _check_segmented(rs, k, v, off, keys_only=True))


@pytest.mark.parametrize("bits", [4, 8])
def test_whole_small_arrays_both_digit_widths(rs, bits):
    """Whole arrays taken by the one-warp sort (up to 512 items) and by the
    one-CTA sort (up to 8192), at digit width 4 and 8."""
    def run():
        for n, dist in ((1, "uniform"), (2, "uniform"), (33, "and2"), (100, "equal"),
                        (512, "uniform"), (513, "low16"), (4096, "and4"), (8192, "uniform"),
                        (8191, "distinct256")):
            k = inputs.keys(dist, n, seed=95)
            v = inputs.index_values(n)
            kd, vd = to_dev(k), to_dev(v)
            rs.sort_pairs(kd, vd)
            ko, vo = oracle.sort_pairs(k, v)
            assert np.array_equal(to_host(kd), ko) and np.array_equal(to_host(vd), vo), (n, dist)
            kd = to_dev(k)
            rs.sort_keys(kd)
            assert np.array_equal(to_host(kd), ko), (n, dist)
    _with_knobs(rs, {"warp_max": 512, "small_max": 8192, "small_bits": bits}, run)


def test_many_tiny_segments_2pow20(rs):
    """2^14 segments with sizes log-uniform on [2, 2^9] (every one on the
    one-warp path): a batch of many short arrays."""
    k, v, off = inputs.segmented_batch(1 << 14, 1, 9, seed=96)
    _check_segmented(rs, k, v, off)
