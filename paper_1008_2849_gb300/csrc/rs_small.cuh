// rs_small.cuh -- sorts of arrays that fit in on-chip memory: the one-warp
// sort (k_warp_sort) and the one-CTA sort (k_small_sort).  Both run the
// stable counting-sort passes of Sec. 3 between two shared-memory buffers, so
// every item is read from and written to global memory once.  The digit width
// BITS is a template parameter: 8 bits (four passes, 256 buckets, as in the
// scatter passes) or 4 bits (eight passes, 16 buckets) -- which is faster
// depends on the array size, and the autotuner picks it per size class.
// Either width gives the same stable order.  Typed keys (key_type) are mapped
// onto their ordered words when read and back when written.  An array is read
// from src_keys / src_vals and written to keys / vals at the same offsets (the
// same arrays for an in-place sort; the other buffer after an MSD pass).
#pragma once

#include "rs_device.cuh"

namespace rs {

constexpr int WARP_SORT_THREADS = 256;  // 8 independent warps per CTA
constexpr int WARP_SORT_ITEMS = 16;     // one warp sorts up to 512 items

// Digit p (BITS wide, p = 0 the least significant) of a key.
template <int BITS>
__device__ __forceinline__ uint32_t small_digit(uint32_t key, uint32_t p) {
    return (key >> (p * BITS)) & ((1u << BITS) - 1u);
}

// Shared words of one warp of k_warp_sort: keys [2][CAP], values [2][CAP]
// (key-value sorts), digit counters [2^BITS].
template <int ITEMS, int BITS, bool PAIRS>
struct WarpSortSmem {
    static constexpr uint32_t CAP = 32 * ITEMS;
    static constexpr uint32_t PER_WARP = (PAIRS ? 4u : 2u) * CAP + (1u << BITS);
    static constexpr size_t BYTES = (size_t)(WARP_SORT_THREADS / 32) * PER_WARP * 4;
};

// ---------------------------------------------------------------------------
// k_warp_sort: every warp sorts whole arrays of at most 32 * ITEMS items, one
// at a time, in its own shared-memory region, with no CTA-wide barrier.
// Arrays are the segments listed in `list` (count ctrl->tiny_count), or with
// off == nullptr the single array [0, single_n).  Per pass: the digit counts
// of the array (shared atomics), their exclusive prefix over digits (each
// lane scans 2^BITS / 32 counters, then a warp scan), then the items slot by
// slot in input order: the lanes holding the same digit come from one ballot
// per digit bit, the lowest of them advances the digit's counter by the
// group's size, and every item goes to the counter's old value plus the
// number of its peers on lower lanes -- a stable counting sort.  A pass whose
// digit is the same for the whole array is skipped.
// ---------------------------------------------------------------------------
template <int ITEMS, int BITS, bool PAIRS>
__global__ void __launch_bounds__(WARP_SORT_THREADS)
k_warp_sort(uint32_t* keys, uint32_t* vals, const uint32_t* src_keys, const uint32_t* src_vals,
            const uint32_t* __restrict__ off, const uint32_t* __restrict__ list,
            const Ctrl* __restrict__ ctrl, uint32_t single_n, uint32_t key_type) {
    using L = WarpSortSmem<ITEMS, BITS, PAIRS>;
    pdl_launch_next();
    pdl_wait();  // the kernel before this one (planner, MSD pass) is complete
    constexpr uint32_t NB = 1u << BITS;
    constexpr uint32_t NPASS = 32 / BITS;
    constexpr uint32_t CAP = L::CAP;
    constexpr uint32_t WARPS = WARP_SORT_THREADS / 32;
    constexpr uint32_t PL = NB >= 32 ? NB / 32 : 1;  // counters scanned per lane
    static_assert(32 % BITS == 0, "whole passes");
    extern __shared__ uint4 s_dyn[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* const s_k = reinterpret_cast<uint32_t*>(s_dyn) + warp * L::PER_WARP;
    uint32_t* const s_v = s_k + 2 * CAP;
    uint32_t* const cnt = s_k + (PAIRS ? 4 : 2) * CAP;
    const uint32_t lt = lanemask_lt();

    uint32_t count = 1;
    if (off != nullptr) {
        if (ctrl->err != 0) return;
        count = ctrl->tiny_count;
    }
    for (uint32_t idx = blockIdx.x * WARPS + warp; idx < count; idx += gridDim.x * WARPS) {
        uint32_t lo = 0, m = single_n;
        if (off != nullptr) {
            const uint32_t s = list[idx];
            lo = off[s];
            m = off[s + 1] - lo;
        }
        for (uint32_t i = lane; i < m; i += 32) {
            s_k[i] = key_to_ordered(src_keys[lo + i], key_type);
            if (PAIRS) s_v[i] = src_vals[lo + i];
        }
        uint32_t cur = 0;
        for (uint32_t p = 0; p < NPASS; ++p) {
            for (uint32_t b = lane; b < NB; b += 32) cnt[b] = 0;
            __syncwarp();
            const uint32_t* ck = s_k + cur * CAP;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((uint32_t)j * 32 >= m) break;  // warp-uniform
                const uint32_t i = j * 32 + lane;
                if (i < m) atomicAdd(&cnt[small_digit<BITS>(ck[i], p)], 1u);
            }
            __syncwarp();
            uint32_t c[PL];
            uint32_t tot = 0;
            bool trivial = false;
#pragma unroll
            for (uint32_t q = 0; q < PL; ++q) {
                const uint32_t d = lane * PL + q;
                c[q] = d < NB ? cnt[d] : 0u;
                trivial |= c[q] == m;
                tot += c[q];
            }
            if (__any_sync(0xffffffffu, trivial)) continue;  // one digit only: identity pass
            uint32_t x = tot;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t run = x - tot;
#pragma unroll
            for (uint32_t q = 0; q < PL; ++q) {
                const uint32_t d = lane * PL + q;
                if (d < NB) cnt[d] = run;
                run += c[q];
            }
            __syncwarp();
            uint32_t* nk = s_k + (cur ^ 1) * CAP;
            const uint32_t* cv = s_v + cur * CAP;
            uint32_t* nv = s_v + (cur ^ 1) * CAP;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((uint32_t)j * 32 >= m) break;  // warp-uniform
                const uint32_t i = j * 32 + lane;
                const uint32_t live = prefix_lanes(j * 32, m);
                const uint32_t k = i < m ? ck[i] : 0u;
                const uint32_t d = small_digit<BITS>(k, p);
                const uint32_t peers = match_label<BITS>(d) & live;
                const uint32_t first = __ffs(peers) - 1;
                uint32_t before = 0;
                if (lane == first) before = atomicAdd(&cnt[d], (uint32_t)__popc(peers));
                before = __shfl_sync(0xffffffffu, before, first & 31u);
                if (i < m) {
                    const uint32_t pos = before + __popc(peers & lt);
                    nk[pos] = k;
                    if (PAIRS) nv[pos] = cv[i];
                }
            }
            __syncwarp();
            cur ^= 1;
        }
        const uint32_t* fk = s_k + cur * CAP;
        const uint32_t* fv = s_v + cur * CAP;
        for (uint32_t i = lane; i < m; i += 32) {
            keys[lo + i] = key_from_ordered(fk[i], key_type);
            if (PAIRS) vals[lo + i] = fv[i];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// k_small_sort: one CTA sorts a whole array of at most CAP = THREADS * ITEMS
// items in shared memory: 32 / BITS stable counting-sort passes between two
// shared buffers.  Arrays are the segments listed in small_list (count in
// ctrl->small_count), or with off == nullptr the single array [0, single_n).
// Per pass: per-warp digit counts, their prefix over (digit, warp), then every
// warp ranks its items slot by slot (peers from one ballot per digit bit,
// positions from the warp's counters) and moves them to the other buffer.  A
// pass whose digit is the same for the whole array is skipped.
// ---------------------------------------------------------------------------
template <int THREADS, int ITEMS, int BITS, bool PAIRS>
__global__ void __launch_bounds__(THREADS)
k_small_sort(uint32_t* keys, uint32_t* vals, const uint32_t* src_keys, const uint32_t* src_vals,
             const uint32_t* __restrict__ off, const uint32_t* __restrict__ small_list,
             const Ctrl* __restrict__ ctrl, uint32_t single_n, uint32_t key_type) {
    constexpr uint32_t NB = 1u << BITS;
    constexpr uint32_t NPASS = 32 / BITS;
    constexpr uint32_t NW = (NB + 31) / 32;  // warps holding digit totals
    constexpr uint32_t WARPS = THREADS / 32;
    constexpr uint32_t CAP = THREADS * ITEMS;
    constexpr uint32_t WARP_ITEMS = 32 * ITEMS;
    static_assert(THREADS >= (int)NB && 32 % BITS == 0, "one thread per digit, whole passes");
    pdl_launch_next();
    pdl_wait();  // the kernel before this one (planner, MSD pass) is complete
    extern __shared__ uint4 s_dyn[];
    uint32_t* const s_k = reinterpret_cast<uint32_t*>(s_dyn);  // [2][CAP]
    uint32_t* const s_v = s_k + 2 * CAP;                       // [2][CAP] (pairs)
    uint32_t* const s_w = s_v + (PAIRS ? 2 * CAP : 0);         // [WARPS][NB]
    __shared__ uint32_t s_scan[NW];
    __shared__ uint32_t s_trivial;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t wofs = warp * WARP_ITEMS;

    uint32_t count = 1;
    if (off != nullptr) {
        if (ctrl->err != 0) return;
        count = ctrl->small_count;
    }
    for (uint32_t w = tid; w < WARPS * NB; w += THREADS) s_w[w] = 0;
    for (uint32_t idx = blockIdx.x; idx < count; idx += gridDim.x) {
        uint32_t lo = 0, m = single_n;
        if (off != nullptr) {
            const uint32_t s = small_list[idx];
            lo = off[s];
            m = off[s + 1] - lo;
        }
        for (uint32_t i = tid; i < m; i += THREADS) {
            s_k[i] = key_to_ordered(src_keys[lo + i], key_type);
            if (PAIRS) s_v[i] = src_vals[lo + i];
        }
        __syncthreads();
        uint32_t cur = 0;
        for (uint32_t p = 0; p < NPASS; ++p) {
            const uint32_t* ck = s_k + cur * CAP;
            uint32_t* row = s_w + warp * NB;
            const uint32_t left = m > wofs ? m - wofs : 0u;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (j * 32 + lane < left) atomicAdd(&row[small_digit<BITS>(ck[wofs + j * 32 + lane], p)], 1u);
            if (tid == 0) s_trivial = 0;
            __syncthreads();
            uint32_t c = 0;
            if (tid < NB) {
#pragma unroll
                for (uint32_t w = 0; w < WARPS; ++w) c += s_w[w * NB + tid];
                if (c == m) s_trivial = 1;
            }
            uint32_t x = c;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (warp < NW && lane == 31) s_scan[warp] = x;
            __syncthreads();
            if (s_trivial) {  // every item has the same digit: the pass is the identity
                for (uint32_t w = tid; w < WARPS * NB; w += THREADS) s_w[w] = 0;
                __syncthreads();
                continue;
            }
            if (tid < NB) {
                uint32_t offv = 0;
                for (uint32_t w = 0; w < warp; ++w) offv += s_scan[w];
                uint32_t run = offv + x - c;
#pragma unroll
                for (uint32_t w = 0; w < WARPS; ++w) {
                    const uint32_t t = s_w[w * NB + tid];
                    s_w[w * NB + tid] = run;
                    run += t;
                }
            }
            __syncthreads();
            uint32_t* nk = s_k + (cur ^ 1) * CAP;
            const uint32_t* cv = s_v + cur * CAP;
            uint32_t* nv = s_v + (cur ^ 1) * CAP;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const uint32_t li = wofs + j * 32 + lane;
                const uint32_t live = prefix_lanes(j * 32, left);
                const uint32_t k = ck[li];
                const uint32_t d = small_digit<BITS>(k, p);
                const uint32_t peers = match_label<BITS>(d) & live;
                const uint32_t first = __ffs(peers) - 1;
                uint32_t before = 0;
                if (lane == first) before = atomicAdd(&row[d], (uint32_t)__popc(peers));
                before = __shfl_sync(0xffffffffu, before, first & 31u);
                if (j * 32 + lane < left) {
                    const uint32_t pos = before + __popc(peers & lt);
                    nk[pos] = k;
                    if (PAIRS) nv[pos] = cv[li];
                }
            }
            __syncwarp();
            for (uint32_t i = lane; i < NB; i += 32) row[i] = 0;
            __syncthreads();
            cur ^= 1;
        }
        const uint32_t* fk = s_k + cur * CAP;
        const uint32_t* fv = s_v + cur * CAP;
        for (uint32_t i = tid; i < m; i += THREADS) {
            keys[lo + i] = key_from_ordered(fk[i], key_type);
            if (PAIRS) vals[lo + i] = fv[i];
        }
        __syncthreads();
    }
}

}  // namespace rs
