/*
 * rs_oracle.c -- CPU oracle for the stable LSD radix sort of 32-bit unsigned
 * keys (optionally carrying a 32-bit value) described by Wassenberg & Sanders,
 * "Faster Radix Sort via Virtual Memory and Write-Combining" (2010).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes, and from which passage:
 *   - Problem statement (Abstract; Sec. 1): 32-bit integer keys, optionally
 *     paired with a 32-bit value.  Keys are read as unsigned and sorted
 *     ascending; a value is an opaque payload that travels with its key.
 *   - One pass = the naive counting sort of Sec. 3: histogram of the digit,
 *     prefix sum to the first output slot of every bucket, then every item in
 *     input order is written at its bucket's slot, which is post-incremented.
 *     Visiting items in input order is what makes the pass stable (Sec. 4).
 *   - The radix sort is the LSD variant of Sec. 4 with K = 32 and D = 8
 *     (Alg. 2 uses D = 8 so that a digit is a byte): K/D = 4 passes over
 *     digits 0 (least significant byte) to 3.  Alg. 2 takes digit 3 first
 *     ("reverse sorting") and then digits 0, 1, 2 inside every MSD bucket;
 *     both orders yield the same unique stable ascending result, and this
 *     oracle uses the plain LSD order.
 *   - Segmented form: the same sort applied to every [off[s], off[s+1]).
 *     The paper has no segmented case; this is the plain definition.
 *   - A threaded variant (per-thread chunk histograms, prefix in
 *     (digit, thread) order, scatter) that yields the identical result; it is
 *     what the CPU baseline times on all host cores.
 *   - 64-bit keys: the same LSD radix sort with K = 64 (Sec. 4 leaves K
 *     general; its experiments use K = 32), D = 8: eight passes over bytes
 *     0..7 of the key, values 32-bit.
 *   - Typed keys (no counterpart in the paper, whose keys are unsigned):
 *     32-bit two's-complement integers ordered by value, and IEEE-754
 *     binary32 floats ordered by the totalOrder predicate of IEEE 754-2008
 *     Sec. 5.10.  These are a plain stable merge sort with that comparison,
 *     written from the definitions, not from any bit transformation.
 *   - Items of every width (Sec. 1: the 32-bit items are a simplification;
 *     larger items sort the same way): 32-bit or 64-bit keys of any of the
 *     types above (64-bit: unsigned, two's-complement, IEEE-754 binary64 by
 *     totalOrder) carrying no, 32-bit or 64-bit values.  Again a plain
 *     stable merge sort with the key comparison; values are opaque bytes.
 *
 * Everything is written as plain loops, with no blocking, fusion or
 * reordering beyond the counting sort itself.
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define RADIX_BITS 8u
#define RADIX 256u
#define PASSES 4u

/* Digit p of a key: byte p, p = 0 least significant (Alg. 2, Digit()). */
static uint32_t digit_of(uint32_t key, unsigned p) {
    return (key >> (RADIX_BITS * p)) & (RADIX - 1u);
}

/* All four digit histograms: hist[p*256 + b] = #{i : digit_of(keys[i], p) == b}.
 * Counting step of the naive counting sort (Sec. 3), done for every digit. */
void oracle_digit_histograms(const uint32_t* keys, size_t n, uint64_t* hist) {
    memset(hist, 0, sizeof(uint64_t) * RADIX * PASSES);
    for (size_t i = 0; i < n; ++i)
        for (unsigned p = 0; p < PASSES; ++p)
            hist[p * RADIX + digit_of(keys[i], p)] += 1;
}

/* Exclusive prefix over the buckets of every digit: first output slot of each
 * bucket (Sec. 3 "prefix sum"; Alg. 2 PrefixSum(bucketSizes)). */
void oracle_exclusive_prefix(const uint64_t* hist, uint64_t* first) {
    for (unsigned p = 0; p < PASSES; ++p) {
        uint64_t run = 0;
        for (unsigned b = 0; b < RADIX; ++b) {
            first[p * RADIX + b] = run;
            run += hist[p * RADIX + b];
        }
    }
}

/* One stable counting-sort pass by digit p (Sec. 3): src -> dst.
 * vals_src / vals_dst may be NULL for keys only. */
void oracle_counting_pass(const uint32_t* keys_src, const uint32_t* vals_src,
                          uint32_t* keys_dst, uint32_t* vals_dst,
                          size_t n, unsigned p) {
    uint64_t count[RADIX];
    uint64_t next[RADIX];
    memset(count, 0, sizeof(count));
    for (size_t i = 0; i < n; ++i)
        count[digit_of(keys_src[i], p)] += 1;
    uint64_t run = 0;
    for (unsigned b = 0; b < RADIX; ++b) {
        next[b] = run;
        run += count[b];
    }
    for (size_t i = 0; i < n; ++i) {
        uint32_t b = digit_of(keys_src[i], p);
        uint64_t slot = next[b];
        next[b] = slot + 1;
        keys_dst[slot] = keys_src[i];
        if (vals_src) vals_dst[slot] = vals_src[i];
    }
}

/* Full LSD radix sort, passes 0..3 (Sec. 4, K = 32, D = 8).
 * keys_out / vals_out receive the result; inputs are not modified.
 * vals_in / vals_out may be NULL (keys only).  Returns 0, or -1 on
 * allocation failure. */
int oracle_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in,
                      uint32_t* keys_out, uint32_t* vals_out, size_t n) {
    if (n == 0) return 0;
    uint32_t* ka = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* kb = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* va = vals_in ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    uint32_t* vb = vals_in ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    if (!ka || !kb || (vals_in && (!va || !vb))) {
        free(ka); free(kb); free(va); free(vb);
        return -1;
    }
    memcpy(ka, keys_in, n * sizeof(uint32_t));
    if (vals_in) memcpy(va, vals_in, n * sizeof(uint32_t));
    for (unsigned p = 0; p < PASSES; ++p) {
        oracle_counting_pass(ka, va, kb, vb, n, p);
        uint32_t* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    memcpy(keys_out, ka, n * sizeof(uint32_t));
    if (vals_in) memcpy(vals_out, va, n * sizeof(uint32_t));
    free(ka); free(kb); free(va); free(vb);
    return 0;
}

/* Segmented sort: every segment [offsets[s], offsets[s+1]) is sorted on its
 * own, s = 0..num_segments-1.  offsets has num_segments + 1 nondecreasing
 * entries; items outside [offsets[0], offsets[S]) are copied unchanged.
 * Returns 0, -1 on allocation failure, -2 on a malformed table. */
int oracle_sort_pairs_segmented(const uint32_t* keys_in, const uint32_t* vals_in,
                                uint32_t* keys_out, uint32_t* vals_out, size_t n,
                                const uint32_t* offsets, uint32_t num_segments) {
    for (uint32_t s = 0; s < num_segments; ++s)
        if (offsets[s] > offsets[s + 1]) return -2;
    if (num_segments > 0 && offsets[num_segments] > n) return -2;
    memcpy(keys_out, keys_in, n * sizeof(uint32_t));
    if (vals_in) memcpy(vals_out, vals_in, n * sizeof(uint32_t));
    for (uint32_t s = 0; s < num_segments; ++s) {
        size_t lo = offsets[s], len = (size_t)offsets[s + 1] - offsets[s];
        int rc = oracle_sort_pairs(keys_in + lo, vals_in ? vals_in + lo : NULL,
                                   keys_out + lo, vals_out ? vals_out + lo : NULL, len);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Threaded variant (same result).  Thread t owns the contiguous chunk
 * [t*n/T, (t+1)*n/T).  Per pass: every thread counts its chunk; the first
 * slot of (bucket b, thread t) is the number of items with a smaller digit
 * plus the items of bucket b held by threads before t; every thread then
 * scatters its chunk in input order.  Since chunks are in input order and
 * slots are assigned in (digit, thread, position) order, the pass is the
 * same stable counting sort as above.
 * ---------------------------------------------------------------------- */
typedef struct {
    size_t lo, hi;                 /* this thread's chunk of the input */
    pthread_barrier_t* bar;
    uint64_t* all_counts;          /* [nthreads][RADIX] chunk histograms */
    unsigned nthreads, tid;
    uint32_t *ka, *kb, *va, *vb;   /* ping-pong buffers shared by all threads */
} par_arg;

static void* par_worker(void* vp) {
    par_arg* a = (par_arg*)vp;
    uint32_t *ks = a->ka, *kd = a->kb, *vs = a->va, *vd = a->vb;
    for (unsigned p = 0; p < PASSES; ++p) {
        uint64_t* mine = a->all_counts + (size_t)a->tid * RADIX;
        memset(mine, 0, RADIX * sizeof(uint64_t));
        for (size_t i = a->lo; i < a->hi; ++i) mine[digit_of(ks[i], p)] += 1;
        pthread_barrier_wait(a->bar);
        uint64_t next[RADIX];
        uint64_t run = 0;
        for (unsigned b = 0; b < RADIX; ++b) {
            for (unsigned t = 0; t < a->nthreads; ++t) {
                if (t == a->tid) next[b] = run;
                run += a->all_counts[(size_t)t * RADIX + b];
            }
        }
        for (size_t i = a->lo; i < a->hi; ++i) {
            uint32_t b = digit_of(ks[i], p);
            uint64_t slot = next[b]++;
            kd[slot] = ks[i];
            if (vs) vd[slot] = vs[i];
        }
        pthread_barrier_wait(a->bar);
        uint32_t* t = ks; ks = kd; kd = t;
        t = vs; vs = vd; vd = t;
    }
    return NULL;
}

int oracle_sort_pairs_threaded(const uint32_t* keys_in, const uint32_t* vals_in,
                               uint32_t* keys_out, uint32_t* vals_out, size_t n,
                               unsigned nthreads) {
    if (n == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    uint32_t* ka = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* kb = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* va = vals_in ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    uint32_t* vb = vals_in ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    uint64_t* counts = (uint64_t*)malloc((size_t)nthreads * RADIX * sizeof(uint64_t));
    par_arg* args = (par_arg*)malloc(nthreads * sizeof(par_arg));
    pthread_t* th = (pthread_t*)malloc(nthreads * sizeof(pthread_t));
    if (!ka || !kb || (vals_in && (!va || !vb)) || !counts || !args || !th) {
        free(ka); free(kb); free(va); free(vb); free(counts); free(args); free(th);
        return -1;
    }
    memcpy(ka, keys_in, n * sizeof(uint32_t));
    if (vals_in) memcpy(va, vals_in, n * sizeof(uint32_t));
    pthread_barrier_t bar;
    pthread_barrier_init(&bar, NULL, nthreads);
    for (unsigned t = 0; t < nthreads; ++t) {
        par_arg* a = &args[t];
        a->lo = (size_t)((unsigned __int128)n * t / nthreads);
        a->hi = (size_t)((unsigned __int128)n * (t + 1) / nthreads);
        a->bar = &bar; a->all_counts = counts; a->nthreads = nthreads; a->tid = t;
        a->ka = ka; a->kb = kb; a->va = va; a->vb = vb;
    }
    for (unsigned t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, par_worker, &args[t]);
    par_worker(&args[0]);
    for (unsigned t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&bar);
    /* PASSES is even, so after the last swap the result is back in ka/va. */
    memcpy(keys_out, ka, n * sizeof(uint32_t));
    if (vals_in) memcpy(vals_out, va, n * sizeof(uint32_t));
    free(ka); free(kb); free(va); free(vb); free(counts); free(args); free(th);
    return 0;
}


/* ------------------------------------------------------------------------
 * Typed keys.  key_type 1: the 32-bit word is a two's-complement integer and
 * keys are ordered by value.  key_type 2: the word is an IEEE-754 binary32
 * and keys are ordered by totalOrder (IEEE 754-2008 Sec. 5.10): every
 * negative-signed encoding before every positive-signed one; among positive
 * signs a larger magnitude (exponent and significand read as one unsigned
 * field) comes later, among negative signs earlier.  This places -NaN before
 * -inf, -0 before +0 and +NaN after +inf, and orders NaNs by payload.
 * Equal keys keep their input order (the merge takes from the left run on
 * ties).
 * ---------------------------------------------------------------------- */
static int typed_less(uint32_t a, uint32_t b, int key_type) {
    if (key_type == 1) return (int32_t)a < (int32_t)b;
    const uint32_t sa = a >> 31, sb = b >> 31;
    const uint32_t ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;
    if (sa != sb) return sa > sb;  /* negative sign first */
    if (sa == 0) return ma < mb;   /* both positive */
    return ma > mb;                /* both negative */
}

static void merge_sort_idx(const uint32_t* keys, uint32_t* idx, uint32_t* tmp, size_t lo,
                           size_t hi, int key_type) {
    if (hi - lo < 2) return;
    const size_t mid = lo + (hi - lo) / 2;
    merge_sort_idx(keys, idx, tmp, lo, mid, key_type);
    merge_sort_idx(keys, idx, tmp, mid, hi, key_type);
    size_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (typed_less(keys[idx[j]], keys[idx[i]], key_type))
            tmp[o++] = idx[j++];
        else
            tmp[o++] = idx[i++];
    }
    while (i < mid) tmp[o++] = idx[i++];
    while (j < hi) tmp[o++] = idx[j++];
    memcpy(idx + lo, tmp + lo, (hi - lo) * sizeof(uint32_t));
}

/* Stable sort of typed keys (key_type 1 or 2; 0 = unsigned, as
 * oracle_sort_pairs).  Returns 0, -1 on allocation failure, -3 on an unknown
 * key type. */
int oracle_sort_typed(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                      uint32_t* vals_out, size_t n, int key_type) {
    if (key_type == 0) return oracle_sort_pairs(keys_in, vals_in, keys_out, vals_out, n);
    if (key_type != 1 && key_type != 2) return -3;
    if (n == 0) return 0;
    uint32_t* idx = (uint32_t*)malloc(n * sizeof(uint32_t));
    uint32_t* tmp = (uint32_t*)malloc(n * sizeof(uint32_t));
    if (!idx || !tmp) {
        free(idx); free(tmp);
        return -1;
    }
    for (size_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
    merge_sort_idx(keys_in, idx, tmp, 0, n, key_type);
    for (size_t i = 0; i < n; ++i) {
        keys_out[i] = keys_in[idx[i]];
        if (vals_in) vals_out[i] = vals_in[idx[i]];
    }
    free(idx); free(tmp);
    return 0;
}

/* Segmented form of oracle_sort_typed (table rules as for
 * oracle_sort_pairs_segmented). */
int oracle_sort_typed_segmented(const uint32_t* keys_in, const uint32_t* vals_in,
                                uint32_t* keys_out, uint32_t* vals_out, size_t n,
                                const uint32_t* offsets, uint32_t num_segments, int key_type) {
    for (uint32_t s = 0; s < num_segments; ++s)
        if (offsets[s] > offsets[s + 1]) return -2;
    if (num_segments > 0 && offsets[num_segments] > n) return -2;
    memcpy(keys_out, keys_in, n * sizeof(uint32_t));
    if (vals_in) memcpy(vals_out, vals_in, n * sizeof(uint32_t));
    for (uint32_t s = 0; s < num_segments; ++s) {
        size_t lo = offsets[s], len = (size_t)offsets[s + 1] - offsets[s];
        int rc = oracle_sort_typed(keys_in + lo, vals_in ? vals_in + lo : NULL, keys_out + lo,
                                   vals_out ? vals_out + lo : NULL, len, key_type);
        if (rc) return rc;
    }
    return 0;
}


/* ------------------------------------------------------------------------
 * 64-bit keys (K = 64, D = 8; Sec. 4): eight stable counting-sort passes,
 * byte 0 (least significant) first, each the naive counting sort of Sec. 3.
 * vals may be NULL.  Returns 0, or -1 on allocation failure.
 * ---------------------------------------------------------------------- */
#define PASSES64 8u

static uint32_t digit64_of(uint64_t key, unsigned p) {
    return (uint32_t)((key >> (RADIX_BITS * p)) & (RADIX - 1u));
}

static void counting_pass64(const uint64_t* keys_src, const uint32_t* vals_src,
                            uint64_t* keys_dst, uint32_t* vals_dst, size_t n, unsigned p) {
    uint64_t count[RADIX];
    uint64_t next[RADIX];
    memset(count, 0, sizeof(count));
    for (size_t i = 0; i < n; ++i)
        count[digit64_of(keys_src[i], p)] += 1;
    uint64_t run = 0;
    for (unsigned b = 0; b < RADIX; ++b) {
        next[b] = run;
        run += count[b];
    }
    for (size_t i = 0; i < n; ++i) {
        uint32_t b = digit64_of(keys_src[i], p);
        uint64_t slot = next[b];
        next[b] = slot + 1;
        keys_dst[slot] = keys_src[i];
        if (vals_src != NULL) vals_dst[slot] = vals_src[i];
    }
}

int oracle_sort_pairs64(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                        uint32_t* vals_out, size_t n) {
    if (n == 0) return 0;
    uint64_t* ka = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t* kb = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint32_t* va = vals_in ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    uint32_t* vb = vals_in ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    if (!ka || !kb || (vals_in && (!va || !vb))) {
        free(ka); free(kb); free(va); free(vb);
        return -1;
    }
    memcpy(ka, keys_in, n * sizeof(uint64_t));
    if (vals_in) memcpy(va, vals_in, n * sizeof(uint32_t));
    for (unsigned p = 0; p < PASSES64; ++p) {
        counting_pass64(ka, va, kb, vb, n, p);
        uint64_t* t = ka; ka = kb; kb = t;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    memcpy(keys_out, ka, n * sizeof(uint64_t));
    if (vals_in) memcpy(vals_out, va, n * sizeof(uint32_t));
    free(ka); free(kb); free(va); free(vb);
    return 0;
}


/* ------------------------------------------------------------------------
 * Keys and values of every width.  key_type 0, 1, 2: 32-bit words read as
 * unsigned, two's-complement or IEEE-754 binary32 (as above); 3, 4, 5: the
 * same three readings of 64-bit words (binary64 totalOrder: sign bit 63,
 * magnitude = the other 63 bits read as one unsigned field).  value_bits 0
 * (keys only), 32 or 64; a value is copied as opaque bytes.  Plain stable
 * merge sort by the key comparison (ties keep input order), then keys and
 * values are gathered in that order.  Returns 0, -1 on allocation failure,
 * -3 on an unknown key_type or value_bits.
 * ---------------------------------------------------------------------- */
static int kv_less(const unsigned char* keys, size_t a, size_t b, int key_type) {
    if (key_type <= 2) {
        uint32_t x, y;
        memcpy(&x, keys + 4 * a, 4);
        memcpy(&y, keys + 4 * b, 4);
        if (key_type == 0) return x < y;
        return typed_less(x, y, key_type);
    }
    uint64_t x, y;
    memcpy(&x, keys + 8 * a, 8);
    memcpy(&y, keys + 8 * b, 8);
    if (key_type == 3) return x < y;
    if (key_type == 4) return (int64_t)x < (int64_t)y;
    const uint64_t sx = x >> 63, sy = y >> 63;
    const uint64_t mx = x & 0x7fffffffffffffffull, my = y & 0x7fffffffffffffffull;
    if (sx != sy) return sx > sy;  /* negative sign first */
    if (sx == 0) return mx < my;   /* both positive */
    return mx > my;                /* both negative */
}

static void merge_sort_kv(const unsigned char* keys, size_t* idx, size_t* tmp, size_t lo,
                          size_t hi, int key_type) {
    if (hi - lo < 2) return;
    const size_t mid = lo + (hi - lo) / 2;
    merge_sort_kv(keys, idx, tmp, lo, mid, key_type);
    merge_sort_kv(keys, idx, tmp, mid, hi, key_type);
    size_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (kv_less(keys, idx[j], idx[i], key_type))
            tmp[o++] = idx[j++];
        else
            tmp[o++] = idx[i++];
    }
    while (i < mid) tmp[o++] = idx[i++];
    while (j < hi) tmp[o++] = idx[j++];
    memcpy(idx + lo, tmp + lo, (hi - lo) * sizeof(size_t));
}

int oracle_sort_kv(const void* keys_in, const void* vals_in, void* keys_out, void* vals_out,
                   size_t n, int key_type, int value_bits) {
    if (key_type < 0 || key_type > 5) return -3;
    if (value_bits != 0 && value_bits != 32 && value_bits != 64) return -3;
    if (n == 0) return 0;
    const size_t kb = key_type <= 2 ? 4 : 8, vb = (size_t)value_bits / 8;
    size_t* idx = (size_t*)malloc(n * sizeof(size_t));
    size_t* tmp = (size_t*)malloc(n * sizeof(size_t));
    if (!idx || !tmp) {
        free(idx); free(tmp);
        return -1;
    }
    for (size_t i = 0; i < n; ++i) idx[i] = i;
    merge_sort_kv((const unsigned char*)keys_in, idx, tmp, 0, n, key_type);
    for (size_t i = 0; i < n; ++i) {
        memcpy((unsigned char*)keys_out + kb * i, (const unsigned char*)keys_in + kb * idx[i], kb);
        if (vb)
            memcpy((unsigned char*)vals_out + vb * i, (const unsigned char*)vals_in + vb * idx[i],
                   vb);
    }
    free(idx); free(tmp);
    return 0;
}
