"""GPU parity tests of the segmented sort of every item width
(rs_sort_kv_segmented_ex): 32-bit and 64-bit keys, unsigned, signed or IEEE
float, carrying no, 32-bit or 64-bit values, every segment sorted on its
own, against the CPU oracle's per-segment stable sort (oracle.sort_kv_segmented),
element by element.

Segment mixes cover empty and one-item segments, segments the one-warp sort
takes (up to 256 items), and segments of one tile, several tiles and many
tiles with ragged ends; segment starts are arbitrary, so most tiles are not
aligned.  Items past the table's last offset must be left untouched, and a
malformed table must be reported with nothing written."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1008_2849_gb300 import inputs

pytestmark = pytest.mark.gpu

KEY_TYPES = ["u32", "i32", "f32", "u64", "i64", "f64"]
VALUE_BITS = [0, 32, 64]


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


def _keys(key_type, n, seed):
    lo = inputs.splitmix32(seed, n, 0)
    if key_type.endswith("32"):
        k = lo
    else:
        hi = inputs.splitmix32(seed, n, 1).astype(np.uint64)
        k = (hi << np.uint64(32)) | lo.astype(np.uint64)
    k = k.copy()
    m = min(k[::7].size, k[3::7].size)
    k[:7 * m:7] = k[3::7][:m]  # equal keys: stability shows through the values
    return k


def _values(bits, n):
    if bits == 0:
        return None
    idx = np.arange(n, dtype=np.uint64)
    if bits == 32:
        return idx.astype(np.uint32)
    return (idx << np.uint64(32)) | (idx ^ np.uint64(0xA5A5A5A5))


def _dev(a):
    import torch
    if a is None:
        return None
    view = np.int64 if a.dtype == np.uint64 else np.int32
    return torch.from_numpy(a.view(view)).cuda()


def _host(t, dtype):
    return t.cpu().numpy().view(dtype)


MIXES = {
    "tiny": [0, 1, 2, 31, 32, 33, 255, 256, 100, 0, 7],
    "mixed": [0, 1, 257, 2688, 2689, 5000, 40_000, 3, 130_001, 0, 77, 9999],
    "large": [300_001, 1, 250_000, 2304 * 3 + 5],
}


@pytest.mark.parametrize("mix", sorted(MIXES))
@pytest.mark.parametrize("value_bits", VALUE_BITS)
@pytest.mark.parametrize("key_type", KEY_TYPES)
def test_kv_segmented_matches_oracle(rs, key_type, value_bits, mix):
    sizes = MIXES[mix]
    off = inputs.offsets_from_sizes(sizes).astype(np.uint32)
    n = int(off[-1]) + 9  # items past the last segment stay where they are
    k = _keys(key_type, n, seed=500 + len(sizes) + value_bits)
    v = _values(value_bits, n)
    kd, vd, od = _dev(k), _dev(v), _dev(off)
    rs.sort_kv_segmented(kd, vd, od, key_type)
    ko, vo = oracle.sort_kv_segmented(k, v, off, key_type)
    assert np.array_equal(_host(kd, k.dtype), ko)
    if v is not None:
        assert np.array_equal(_host(vd, v.dtype), vo)


def test_kv_segmented_many_short_segments(rs):
    """Tens of thousands of segments of 0..300 items (one-warp sorts and
    single-tile scatter segments side by side), 64-bit keys and values."""
    sizes = (inputs.splitmix32(510, 30_000, 0) % np.uint32(301)).astype(np.int64)
    off = inputs.offsets_from_sizes(sizes).astype(np.uint32)
    n = int(off[-1])
    k = _keys("i64", n, seed=511)
    v = _values(64, n)
    kd, vd, od = _dev(k), _dev(v), _dev(off)
    rs.sort_kv_segmented(kd, vd, od, "i64")
    ko, vo = oracle.sort_kv_segmented(k, v, off, "i64")
    assert np.array_equal(_host(kd, np.uint64), ko) and np.array_equal(_host(vd, np.uint64), vo)


def test_kv_segmented_bad_table(rs):
    """A decreasing table: RS_ERR_BAD_SEGMENTS, and the data is untouched."""
    off = np.array([0, 500, 400, 900], dtype=np.uint32)
    k = _keys("u64", 1000, seed=520)
    v = _values(64, 1000)
    kd, vd, od = _dev(k), _dev(v), _dev(off)
    with pytest.raises(rs.RsError) as ei:
        rs.sort_kv_segmented(kd, vd, od, "u64")
    assert ei.value.code == 7
    assert rs.stream_status() == 0
    assert np.array_equal(_host(kd, np.uint64), k) and np.array_equal(_host(vd, np.uint64), v)


def test_kv_segmented_workspace_and_args(rs):
    import torch
    assert rs.workspace_bytes_kv_segmented(0, "u64", 64, 3) == 0
    assert rs.workspace_bytes_kv_segmented(1000, "u64", 64, 0) == 0
    w = rs.workspace_bytes_kv_segmented(10_000, "f64", 64, 10)
    assert w >= rs.workspace_bytes_kv(10_000, "f64", 64)
    kd = torch.zeros(100, dtype=torch.int64, device="cuda")
    od = torch.tensor([0, 50, 100], dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    # Values given for a keys-only sort, and none for a key-value sort.
    assert rs.lib().rs_sort_kv_segmented_ex(kd.data_ptr(), kd.data_ptr(), 100, od.data_ptr(), 2,
                                            3, 0, None, ws.data_ptr(), ws.numel()) == 1
    assert rs.lib().rs_sort_kv_segmented_ex(kd.data_ptr(), None, 100, od.data_ptr(), 2, 3, 64,
                                            None, ws.data_ptr(), ws.numel()) == 1
    # A workspace that is too small.
    assert rs.lib().rs_sort_kv_segmented_ex(kd.data_ptr(), None, 100, od.data_ptr(), 2, 3, 0,
                                            None, ws.data_ptr(), 16) == 1
