"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each ``pin_*`` function raises AssertionError when the oracle (the default
build, or a library bound from a mutated copy of its C source) disagrees with
something other than itself:

* numpy's stable argsort (a library routine with the same unique answer),
* the closed-form stable rank  rank(i) = #{j : k_j < k_i} + #{j < i : k_j = k_i}
  evaluated by brute force on tiny inputs and exhaustively on small alphabets,
* invariants (nondecreasing, permutation, equal keys keep input order),
* special cases with known answers (all equal, sorted, reverse sorted),
* closed-form histograms and prefix sums.

The paper defines a pass as the naive counting sort of Sec. 3, the sort as
LSD radix with K = 32 and D = 8 (Sec. 4, Alg. 2), and stability as keeping
the input order of equal keys (Sec. 4).
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle
from paper_1008_2849_gb300 import inputs


def stable_rank_bruteforce(keys):
    """rank(i) = #{j : k_j < k_i} + #{j < i : k_j == k_i}, by plain loops."""
    n = len(keys)
    rank = [0] * n
    for i in range(n):
        r = 0
        for j in range(n):
            if keys[j] < keys[i] or (keys[j] == keys[i] and j < i):
                r += 1
        rank[i] = r
    return rank


def pin_numpy_stable(lib=None):
    cases = [("uniform", 1), ("uniform", 2), ("uniform", 31), ("uniform", 4097),
             ("uniform", 100003), ("and2", 65537), ("and4", 50000),
             ("distinct256", 70001), ("low16", 30011), ("equal", 1000),
             ("sorted", 5000), ("reverse", 5000)]
    for dist, n in cases:
        k = inputs.keys(dist, n, seed=7)
        v = inputs.index_values(n)
        ko, vo = oracle.sort_pairs(k, v, lib=lib)
        perm = np.argsort(k, kind="stable")
        assert np.array_equal(ko, k[perm]), (dist, n, "keys")
        assert np.array_equal(vo, v[perm]), (dist, n, "values")
        kk = oracle.sort_keys(k, lib=lib)
        assert np.array_equal(kk, k[perm]), (dist, n, "keys only")


def pin_bruteforce_tiny(lib=None):
    rng_keys = [inputs.splitmix32(5, n, 0) for n in (0, 1, 2, 3, 7, 16, 33)]
    # Small alphabets force many ties, where stability is visible.
    rng_keys += [inputs.splitmix32(6, 40, 0) & np.uint32(0x03000301)]
    for k in rng_keys:
        n = k.size
        v = inputs.splitmix32(8, n, 1)  # arbitrary payloads
        ko, vo = oracle.sort_pairs(k, v, lib=lib)
        rank = stable_rank_bruteforce([int(x) for x in k])
        exp_k = np.empty_like(k)
        exp_v = np.empty_like(v)
        for i in range(n):
            exp_k[rank[i]] = k[i]
            exp_v[rank[i]] = v[i]
        assert np.array_equal(ko, exp_k), ("keys", n)
        assert np.array_equal(vo, exp_v), ("values", n)


# Four-symbol alphabets: each puts its order into different bytes, so a pass
# that is dropped, reordered or mis-shifted, or a signed reading, shows up.
ALPHABETS = (
    (0x00000001, 0x00000100, 0x00010000, 0x01000000),
    (0xFF000000, 0x00FFFFFF, 0x80000000, 0x7FFFFFFF),
    (0x00000102, 0x00000201, 0x00000101, 0x00000202),
    (0x01FF00FF, 0x0100FF00, 0x00FFFF00, 0x0000FFFF),
)


def pin_exhaustive_small(lib=None, max_len=6):
    """Every sequence of length <= max_len over each alphabet, as segments."""
    for alpha in ALPHABETS:
        seqs = []
        for L in range(0, max_len + 1):
            seqs.extend(itertools.product(range(4), repeat=L))
        sizes = np.array([len(s) for s in seqs], dtype=np.uint64)
        off = inputs.offsets_from_sizes(sizes)
        sym = np.fromiter(itertools.chain.from_iterable(seqs), dtype=np.int64,
                          count=int(off[-1]))
        k = np.asarray(alpha, dtype=np.uint32)[sym]
        v = np.arange(k.size, dtype=np.uint32)
        ko, vo = oracle.sort_pairs_segmented(k, v, off, lib=lib)
        # Expected: per segment, stable rank by the closed form, vectorised
        # over all segments of one length at a time.
        for L in range(1, max_len + 1):
            idx = np.nonzero(sizes == L)[0]
            starts = off[idx].astype(np.int64)
            cols = starts[:, None] + np.arange(L)[None, :]
            kk = k[cols].astype(np.int64)                    # (S, L)
            less = (kk[:, None, :] < kk[:, :, None]).sum(axis=2)
            tri = np.tril(np.ones((L, L), dtype=bool), -1)   # j < i
            eq_before = ((kk[:, None, :] == kk[:, :, None]) & tri[None]).sum(axis=2)
            rank = less + eq_before                          # (S, L)
            exp_k = np.empty_like(kk)
            exp_v = np.empty_like(kk)
            rows = np.arange(len(idx))[:, None]
            exp_k[rows, rank] = kk
            exp_v[rows, rank] = cols
            assert np.array_equal(ko[cols].astype(np.int64), exp_k), (alpha, L, "keys")
            assert np.array_equal(vo[cols].astype(np.int64), exp_v), (alpha, L, "values")


def pin_invariants(lib=None):
    for dist in inputs.DISTRIBUTIONS:
        n = 20011
        k = inputs.keys(dist, n, seed=11)
        v = inputs.index_values(n)
        ko, vo = oracle.sort_pairs(k, v, lib=lib)
        assert np.all(ko[1:] >= ko[:-1]), (dist, "nondecreasing")
        assert np.array_equal(np.sort(vo), v), (dist, "values form a permutation")
        assert np.array_equal(k[vo], ko), (dist, "each key travels with its value")
        same = ko[1:] == ko[:-1]
        assert np.all(vo[1:][same] > vo[:-1][same]), (dist, "stable")


def pin_special_cases(lib=None):
    n = 9999
    v = inputs.index_values(n)
    # All keys equal: identity permutation.
    ko, vo = oracle.sort_pairs(inputs.keys("equal", n, 3), v, lib=lib)
    assert np.array_equal(vo, v)
    # Already sorted: identity permutation.
    k = inputs.keys("sorted", n, 4)
    ko, vo = oracle.sort_pairs(k, v, lib=lib)
    assert np.array_equal(vo, v) and np.array_equal(ko, k)
    # Reverse sorted with distinct keys: the permutation is the reversal.
    k = np.arange(n, 0, -1, dtype=np.uint32) * np.uint32(429497)
    ko, vo = oracle.sort_pairs(k, v, lib=lib)
    assert np.array_equal(vo, v[::-1]) and np.array_equal(ko, k[::-1])
    # Keys 0..n-1 in a fixed shuffled order come out as 0..n-1.
    perm = np.argsort(inputs.splitmix32(9, n, 0), kind="stable").astype(np.uint32)
    ko, vo = oracle.sort_pairs(perm, v, lib=lib)
    assert np.array_equal(ko, v) and np.array_equal(perm[vo], v)
    # Top bit set sorts after top bit clear (unsigned keys, Abstract / Sec. 1).
    k = np.array([0x80000000, 0x7FFFFFFF, 0xFFFFFFFF, 0], dtype=np.uint32)
    ko, _ = oracle.sort_pairs(k, None, lib=lib)
    assert ko.tolist() == [0, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF]


def pin_histograms(lib=None):
    # Keys 0..65535: bytes 0 and 1 take every value 256 times, bytes 2 and 3
    # are always zero.
    k = np.arange(65536, dtype=np.uint32)
    h = oracle.digit_histograms(k, lib=lib)
    assert np.all(h[0] == 256) and np.all(h[1] == 256)
    assert h[2, 0] == 65536 and h[2, 1:].sum() == 0
    assert h[3, 0] == 65536 and h[3, 1:].sum() == 0
    # Against numpy's bincount of each byte.
    k = inputs.keys("and2", 54321, 12)
    h = oracle.digit_histograms(k, lib=lib)
    for p in range(4):
        ref = np.bincount((k >> np.uint32(8 * p)) & np.uint32(255), minlength=256)
        assert np.array_equal(h[p], ref.astype(np.uint64)), p
    # Prefix: closed form on flat counts, and numpy's cumsum otherwise.
    g = oracle.exclusive_prefix(np.full((4, 256), 3, dtype=np.uint64), lib=lib)
    assert np.array_equal(g, np.tile(np.arange(256, dtype=np.uint64) * 3, (4, 1)))
    g = oracle.exclusive_prefix(h, lib=lib)
    ref = np.concatenate([np.zeros((4, 1), dtype=np.uint64), np.cumsum(h, axis=1)[:, :-1]], axis=1)
    assert np.array_equal(g, ref)


def pin_counting_pass(lib=None):
    k = inputs.keys("uniform", 30001, 13)
    v = inputs.index_values(k.size)
    for p in range(4):
        ko, vo = oracle.counting_pass(k, v, p, lib=lib)
        d = (k >> np.uint32(8 * p)) & np.uint32(255)
        perm = np.argsort(d, kind="stable")
        assert np.array_equal(ko, k[perm]) and np.array_equal(vo, v[perm]), p


def pin_segmented(lib=None):
    sizes = np.array([0, 1, 5, 0, 300, 1, 4096, 2, 0, 777], dtype=np.uint64)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    k = inputs.keys("and2", n, 14)
    v = inputs.index_values(n)
    ko, vo = oracle.sort_pairs_segmented(k, v, off, lib=lib)
    for s in range(sizes.size):
        a, b = int(off[s]), int(off[s + 1])
        perm = np.argsort(k[a:b], kind="stable")
        assert np.array_equal(ko[a:b], k[a:b][perm]), s
        assert np.array_equal(vo[a:b], v[a:b][perm]), s


def pin_threaded(lib=None):
    for n in (1, 3, 1000, 65537):
        k = inputs.keys("and3", n, 15)
        v = inputs.index_values(n)
        ref_k, ref_v = oracle.sort_pairs(k, v, lib=lib)
        for t in (1, 2, 3, 8):
            ko, vo = oracle.sort_pairs_threaded(k, v, t, lib=lib)
            assert np.array_equal(ko, ref_k) and np.array_equal(vo, ref_v), (n, t)


# ---------------------------------------------------------------------------
# Typed keys: signed 32-bit integers by value; IEEE-754 binary32 by the
# totalOrder predicate (IEEE 754-2008 Sec. 5.10).  The paper's keys are
# unsigned; these pins fix the typed oracle against numpy and against the
# standard's own listing of the order.
# ---------------------------------------------------------------------------
def _golden_float_order():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "float_total_order.txt")
    words = []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            words.append(int(line.split()[0], 16))
    return np.array(words, dtype=np.uint32)


def pin_typed_i32_numpy(lib=None):
    """Signed keys: numpy's stable argsort of the int32 view, with extremes
    and many duplicates."""
    k = inputs.keys("uniform", 5000, seed=31)
    k[::7] = inputs.keys("distinct256", k[::7].size, seed=32)
    k[:6] = np.array([0x80000000, 0x7FFFFFFF, 0xFFFFFFFF, 0, 1, 0x80000001], dtype=np.uint32)
    v = inputs.index_values(k.size)
    ko, vo = oracle.sort_typed(k, v, "i32", lib=lib)
    order = np.argsort(k.view(np.int32), kind="stable")
    assert np.array_equal(vo, v[order]) and np.array_equal(ko, k[order])


def pin_typed_f32_numpy(lib=None):
    """Float keys without NaNs or zeros (numpy orders those differently from
    totalOrder): numpy's stable argsort of the float32 view, across signs,
    magnitudes from subnormal to infinity, and duplicates."""
    u = inputs.keys("uniform", 6000, seed=33)
    exp = (u >> np.uint32(24)) % np.uint32(255)          # never the NaN exponent 255
    k = (u & np.uint32(0x807FFFFF)) | (exp << np.uint32(23))
    k[::5] = k[1::5][: k[::5].size]                       # duplicates
    k[:4] = np.array([0xFF800000, 0x7F800000, 0x00000001, 0x80000001], dtype=np.uint32)
    k[(k & np.uint32(0x7FFFFFFF)) == 0] = 0x3F800000      # no zeros
    v = inputs.index_values(k.size)
    ko, vo = oracle.sort_typed(k, v, "f32", lib=lib)
    order = np.argsort(k.view(np.float32), kind="stable")
    assert np.array_equal(vo, v[order]) and np.array_equal(ko, k[order])


def pin_typed_f32_total_order(lib=None):
    """The listed totalOrder sequence, shuffled, comes back in that order."""
    want = _golden_float_order()
    for seed in (34, 35, 36):
        perm = np.argsort(inputs.uniform01(seed, want.size, 0), kind="stable")
        ko, _ = oracle.sort_typed(want[perm], None, "f32", lib=lib)
        assert np.array_equal(ko, want)


def pin_typed_stability(lib=None):
    """Equal keys (including repeated -0 and NaN words) keep input order."""
    base = _golden_float_order()
    idx = inputs.splitmix32(37, 3000, 0) % np.uint32(base.size)
    k = base[idx]
    v = inputs.index_values(k.size)
    for kt in ("f32", "i32"):
        ko, vo = oracle.sort_typed(k, v, kt, lib=lib)
        same = ko[1:] == ko[:-1]
        assert np.all(vo[1:][same] > vo[:-1][same])
        assert np.array_equal(np.sort(vo), v)


def pin_typed_segmented(lib=None):
    """Segmented typed sort = the typed sort of every segment on its own."""
    k = inputs.keys("uniform", 3000, seed=38)
    v = inputs.index_values(k.size)
    off = inputs.offsets_from_sizes([0, 1, 700, 2, 1500, 0, 797])
    for kt in ("i32", "f32"):
        ko, vo = oracle.sort_typed_segmented(k, v, off, kt, lib=lib)
        for a, b in zip(off[:-1], off[1:]):
            ek, ev = oracle.sort_typed(k[a:b], v[a:b], kt, lib=lib)
            assert np.array_equal(ko[a:b], ek) and np.array_equal(vo[a:b], ev)


# ---------------------------------------------------------------------------
# 64-bit keys (K = 64, D = 8: eight passes, Sec. 4).
# ---------------------------------------------------------------------------
def _keys64(n, seed):
    hi = inputs.splitmix32(seed, n, 0).astype(np.uint64)
    lo = inputs.splitmix32(seed, n, 1).astype(np.uint64)
    return (hi << np.uint64(32)) | lo


def pin_sort64_numpy(lib=None):
    """numpy's stable argsort of uint64 keys: random words, keys equal in the
    low word only, keys equal in the high word only, and repeats."""
    n = 6000
    k = _keys64(n, 41)
    k[::3] = (k[::3] & np.uint64(0xFFFFFFFF00000000)) | np.uint64(7)        # shared low word
    k[1::5] = (k[1::5] & np.uint64(0xFFFFFFFF)) | np.uint64(0x5 << 40)       # shared high word
    k[2::7] = k[0]
    v = inputs.index_values(n)
    ko, vo = oracle.sort_pairs64(k, v, lib=lib)
    order = np.argsort(k, kind="stable")
    assert np.array_equal(ko, k[order]) and np.array_equal(vo, v[order])


def pin_sort64_bruteforce(lib=None):
    """The closed-form stable rank on tiny arrays whose keys differ only in
    the top byte, only in byte 4, or only in the bottom byte."""
    for shift in (56, 32, 0):
        for seed in range(3):
            raw = inputs.splitmix32(50 + seed, 9, 0) % np.uint32(4)
            k = raw.astype(np.uint64) << np.uint64(shift)
            v = inputs.index_values(k.size)
            ko, vo = oracle.sort_pairs64(k, v, lib=lib)
            rank = stable_rank_bruteforce(k.tolist())
            want_v = np.empty_like(v)
            want_v[rank] = v
            assert np.array_equal(vo, want_v) and np.array_equal(ko, k[vo])


KEY64_PINS = (pin_sort64_numpy, pin_sort64_bruteforce)


# ---------------------------------------------------------------------------
# Items of every width (Sec. 1: larger items sort like the 32-bit ones): keys
# u32, i32, f32, u64, i64, f64 with no, 32-bit or 64-bit values.  Pinned
# against numpy's stable argsort of the typed view, the standard's listing of
# the binary64 totalOrder, the brute-force stable rank, and the radix-sort
# oracles above (an independent algorithm with the same unique answer).
# ---------------------------------------------------------------------------
def _golden_double_order():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "double_total_order.txt")
    words = []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            words.append(int(line.split()[0], 16))
    return np.array(words, dtype=np.uint64)


def _values64(n):
    """Index-derived 64-bit payloads whose halves differ: a value carried
    only in part, or from the wrong item, shows."""
    i = np.arange(n, dtype=np.uint64)
    return (i ^ np.uint64(0xA5A5A5A5)) << np.uint64(32) | i


def _kv_keys(key_type, n, seed):
    """Keys of every reading: random words with duplicates and extremes;
    float keys without NaNs and zeros (numpy orders those apart from
    totalOrder; the golden listings cover them)."""
    if key_type.endswith("32"):
        k = inputs.keys("uniform", n, seed)
        k[::6] = k[1::6][: k[::6].size]
        if key_type == "f32":
            exp = (k >> np.uint32(24)) % np.uint32(255)
            k = (k & np.uint32(0x807FFFFF)) | (exp << np.uint32(23))
            k[(k & np.uint32(0x7FFFFFFF)) == 0] = 0x3F800000
        return k
    k = _keys64(n, seed)
    k[::6] = k[1::6][: k[::6].size]
    k[:4] = np.array([0, 0x7FFFFFFFFFFFFFFF, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
    if key_type == "f64":
        exp = (k >> np.uint64(52)) % np.uint64(2047)         # never the NaN exponent 2047
        k = (k & np.uint64(0x800FFFFFFFFFFFFF)) | (exp << np.uint64(52))
        k[(k & np.uint64(0x7FFFFFFFFFFFFFFF)) == 0] = 0x3FF0000000000000
    return k


_NUMPY_VIEW = {"u32": np.uint32, "i32": np.int32, "f32": np.float32,
               "u64": np.uint64, "i64": np.int64, "f64": np.float64}


def pin_kv_numpy(lib=None):
    """Every key type with no, 32-bit and 64-bit values: numpy's stable
    argsort of the typed view."""
    n = 3000
    for i, kt in enumerate(_NUMPY_VIEW):
        k = _kv_keys(kt, n, seed=60 + i)
        order = np.argsort(k.view(_NUMPY_VIEW[kt]), kind="stable")
        for v in (None, inputs.index_values(n), _values64(n)):
            ko, vo = oracle.sort_kv(k, v, kt, lib=lib)
            assert np.array_equal(ko, k[order])
            if v is not None:
                assert np.array_equal(vo, v[order])


def pin_kv_double_total_order(lib=None):
    """The listed binary64 totalOrder sequence, shuffled, comes back in that
    order.  The listing itself is checked against numpy's float64 reading of
    its non-NaN words (ascending, -0 and +0 equal)."""
    want = _golden_double_order()
    f = want.view(np.float64)
    finite = ~np.isnan(f)
    assert np.all(np.diff(f[finite]) >= 0)
    assert np.count_nonzero(np.diff(f[finite]) == 0) == 1        # only -0, +0
    for seed in (61, 62, 63):
        perm = np.argsort(inputs.uniform01(seed, want.size, 0), kind="stable")
        ko, vo = oracle.sort_kv(want[perm], _values64(want.size), "f64", lib=lib)
        assert np.array_equal(ko, want)
        assert np.array_equal(vo, _values64(want.size)[np.argsort(perm)])


def pin_kv_bruteforce(lib=None):
    """The closed-form stable rank on tiny arrays over small alphabets of
    each reading (signed values straddling zero, floats of both signs)."""
    alphabets = {
        "i64": [0xFFFFFFFFFFFFFFFF, 0, 1, 0x8000000000000000, 0x7FFFFFFFFFFFFFFF],
        "u64": [0xFFFFFFFFFFFFFFFF, 0, 1, 0x8000000000000000, 0x7FFFFFFFFFFFFFFF],
        "f64": [0xBFF0000000000000, 0x3FF0000000000000, 0xC000000000000000,
                0x0000000000000001, 0x8000000000000001],
        "i32": [0xFFFFFFFF, 0, 1, 0x80000000, 0x7FFFFFFF],
    }
    for kt, alpha in alphabets.items():
        dt = np.uint64 if kt.endswith("64") else np.uint32
        for seed in range(4):
            pick = inputs.splitmix32(70 + seed, 9, 0) % np.uint32(len(alpha))
            k = np.array([alpha[i] for i in pick], dtype=dt)
            vals = k.view(_NUMPY_VIEW[kt]).tolist()
            rank = stable_rank_bruteforce(vals)
            v = _values64(k.size)
            ko, vo = oracle.sort_kv(k, v, kt, lib=lib)
            want_v = np.empty_like(v)
            want_v[rank] = v
            assert np.array_equal(vo, want_v)
            want_k = np.empty_like(k)
            want_k[rank] = k
            assert np.array_equal(ko, want_k)


def pin_kv_radix_oracles(lib=None):
    """Unsigned keys: the merge sort agrees with the LSD radix-sort oracles
    (32-bit keys, 64-bit keys with 32-bit values) and carries 64-bit values
    along the same permutation as 32-bit ones."""
    n = 5000
    k32 = _kv_keys("u32", n, seed=80)
    k64 = _kv_keys("u64", n, seed=81)
    v32 = inputs.index_values(n)
    ko, vo = oracle.sort_kv(k32, v32, "u32", lib=lib)
    rk, rv = oracle.sort_pairs(k32, v32)
    assert np.array_equal(ko, rk) and np.array_equal(vo, rv)
    ko, vo = oracle.sort_kv(k64, v32, "u64", lib=lib)
    rk, rv = oracle.sort_pairs64(k64, v32)
    assert np.array_equal(ko, rk) and np.array_equal(vo, rv)
    _, wide = oracle.sort_kv(k64, _values64(n), "u64", lib=lib)
    assert np.array_equal(wide, _values64(n)[rv])


def pin_kv_segmented(lib=None):
    """Segmented sort of every key type with 64-bit values: numpy's stable
    argsort of the typed view inside each segment (empty and one-item
    segments included); items outside the table's range are unchanged."""
    sizes = [0, 1, 700, 2, 1500, 0, 797, 3]
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1]) + 5  # five items past the last segment
    for i, kt in enumerate(_NUMPY_VIEW):
        k = _kv_keys(kt, n, seed=90 + i)
        v = _values64(n)
        ko, vo = oracle.sort_kv_segmented(k, v, off, kt, lib=lib)
        for a, b in zip(off[:-1], off[1:]):
            order = np.argsort(k[a:b].view(_NUMPY_VIEW[kt]), kind="stable")
            assert np.array_equal(ko[a:b], k[a:b][order])
            assert np.array_equal(vo[a:b], v[a:b][order])
        assert np.array_equal(ko[off[-1]:], k[off[-1]:]) and np.array_equal(vo[off[-1]:], v[off[-1]:])


KV_PINS = (pin_kv_numpy, pin_kv_double_total_order, pin_kv_bruteforce, pin_kv_radix_oracles,
           pin_kv_segmented)

TYPED_PINS = (pin_typed_i32_numpy, pin_typed_f32_numpy, pin_typed_f32_total_order,
              pin_typed_stability, pin_typed_segmented)

ALL_PINS = (pin_numpy_stable, pin_bruteforce_tiny, pin_exhaustive_small, pin_invariants,
            pin_special_cases, pin_histograms, pin_counting_pass, pin_segmented,
            pin_threaded)
