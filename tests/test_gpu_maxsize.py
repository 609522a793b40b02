"""The largest arrays the C ABI takes: n = 2^32 - 1 items (keys only and
key-value pairs), so every 32-bit position, tile index and bucket offset
runs up to its limit and the look-back uses 64-bit status words.  Too large
for the CPU oracle, so the results are checked on the device, chunk by
chunk, through properties that fix the unique stable sort:
  - keys nondecreasing (across chunk boundaries too);
  - keys only: the four digit histograms of input and output are equal, and
    so are order-independent sums of the keys (a necessary condition of
    being the same multiset, checked in 64-bit arithmetic);
  - pairs (value = input index): every value appears once, each key is the
    input key at its value, and equal keys keep increasing values."""
from __future__ import annotations

import pytest

from paper_1008_2849_gb300 import inputs

pytestmark = pytest.mark.gpu

N = (1 << 32) - 1
CHUNK = 1 << 28
MASK = 0xFFFFFFFF


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1008_2849_gb300 import build, rs as _rs
    build.build_library()
    _rs.lib()
    return _rs


def _draw(torch, seed):
    k = torch.empty(N, dtype=torch.int32, device="cuda")
    for c in range(0, N, CHUNK):
        m = min(CHUNK, N - c)
        inputs.splitmix32_torch(seed, m, 0, start=c, out=k[c:c + m])
    return k


def _nondecreasing(torch, k):
    for c in range(0, N, CHUNK):
        m = min(CHUNK + 1, N - c)      # one item of overlap with the next chunk
        u = k[c:c + m].to(torch.int64) & MASK
        assert bool((u[1:] >= u[:-1]).all()), c
        del u


def _sums(torch, k):
    s1 = torch.zeros((), dtype=torch.int64, device="cuda")
    s2 = torch.zeros((), dtype=torch.int64, device="cuda")
    for c in range(0, N, CHUNK):
        u = k[c:c + CHUNK].to(torch.int64) & MASK
        s1 += u.sum()
        s2 += (u * u).sum()            # wraps modulo 2^64: still order-independent
        del u
    return int(s1), int(s2)


def test_keys_max_size(rs):
    import torch
    k = _draw(torch, 300)
    h_in = rs.digit_histograms(k).clone()
    s_in = _sums(torch, k)
    rs.sort_keys(k)
    _nondecreasing(torch, k)
    assert torch.equal(rs.digit_histograms(k), h_in)
    assert _sums(torch, k) == s_in
    del k
    torch.cuda.empty_cache()


def test_pairs_max_size(rs):
    import torch
    k = _draw(torch, 301)
    orig = k.clone()
    v = torch.empty(N, dtype=torch.int32, device="cuda")
    for c in range(0, N, CHUNK):
        m = min(CHUNK, N - c)
        v[c:c + m] = torch.arange(c, c + m, dtype=torch.int64, device="cuda").to(torch.int32)
    rs.sort_pairs(k, v)
    _nondecreasing(torch, k)
    seen = torch.zeros(N, dtype=torch.bool, device="cuda")
    for c in range(0, N, CHUNK):
        m = min(CHUNK + 1, N - c)
        vi = v[c:c + m].to(torch.int64) & MASK
        # Range first: indexing by an out-of-range value would be a device-side error.
        assert bool((vi < N).all()), c
        ku = k[c:c + m].to(torch.int64) & MASK
        assert bool(((orig[vi].to(torch.int64) & MASK) == ku).all()), c
        same = ku[1:] == ku[:-1]
        assert bool((vi[1:][same] > vi[:-1][same]).all()), c
        seen[vi[:min(CHUNK, m)]] = True
        del vi, ku, same
    assert bool(seen.all())
    del k, v, orig, seen
    torch.cuda.empty_cache()


def test_digits11_keys_max_size(rs):
    """The 11/11/10-bit sort at n = 2^32 - 1 keys (two alternate buffers of
    16 GiB in the workspace; chunk offsets, tile bases and output slots at
    their 32-bit limits)."""
    import torch
    k = _draw(torch, 302)
    h_in = rs.digit_histograms(k).clone()
    s_in = _sums(torch, k)
    ws = rs.alloc_workspace_digits11(N, False)
    rs.sort_digits11_ex(k, None, ws)
    rs.check_stream()
    del ws
    _nondecreasing(torch, k)
    assert torch.equal(rs.digit_histograms(k), h_in)
    assert _sums(torch, k) == s_in
    del k
    torch.cuda.empty_cache()
