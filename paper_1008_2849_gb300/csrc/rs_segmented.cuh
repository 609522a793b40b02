// rs_segmented.cuh -- kernels of the segmented sort and of the one-CTA sort.
//
// A segmented sort sorts every segment [off[s], off[s+1]) of one array on its
// own (the paper has no segmented case; this is the plain definition applied
// per segment).  Segments are routed by size:
//   small (2 <= size <= small_max): k_small_sort, one CTA per segment, the
//       whole segment in shared memory for all four passes -- one read and one
//       write of every item;
//   large (size > small_max): the scatter passes of the unsegmented sort
//       (k_onesweep<..., SEG>) over tiles that never straddle a segment, after
//       k_seg_hist (per-segment digit histograms) and k_seg_scan (per-segment
//       bucket bases).
// k_seg_plan validates the table and lays the work out.
#pragma once

#include "rs_device.cuh"

namespace rs {

// ---------------------------------------------------------------------------
// k_seg_plan: one CTA of 1024 threads.
//  - Validates the table: nondecreasing, off[S] <= n, every segment < 2^30
//    items.  A bad table sets ERR_SEGMENTS; every later kernel then exits
//    without writing anything.
//  - Large segments get consecutive tile ids (in segment order) and a dense
//    ordinal; tile_geo[t] = (first item, item count, first tile of its
//    segment, ordinal of its segment).
//  - Small segments are listed in small_list (order irrelevant).
//  - The pass plan runs all four passes (caller -> alternate -> ... -> caller).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_seg_plan(const uint32_t* __restrict__ off, uint32_t num_segments, uint32_t n, uint32_t tile,
           uint32_t small_max, Ctrl* __restrict__ ctrl, uint32_t* __restrict__ sticky,
           uint4* __restrict__ tile_geo, uint32_t* __restrict__ small_list,
           uint32_t* __restrict__ large_first /* [S] first item of large ordinal */) {
    __shared__ uint32_t s_carry[2];  // tiles and large segments before this chunk
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    bool bad = false;
    for (uint32_t s = tid; s < num_segments; s += 1024) {
        const uint32_t a = off[s], b = off[s + 1];
        if (b < a || b - a >= (1u << 30)) bad = true;
    }
    if (tid == 0 && off[num_segments] > n) bad = true;
    if (__syncthreads_or(bad)) {
        if (tid == 0) record_error(ctrl, sticky, ERR_SEGMENTS);
        return;
    }
    if (tid == 0) {
        s_carry[0] = 0;
        s_carry[1] = 0;
        for (uint32_t p = 0; p < PASSES; ++p) ctrl->dir[p] = (p & 1) ? DIR_B_TO_A : DIR_A_TO_B;
    }
    __syncthreads();
    for (uint32_t c = 0; c < num_segments; c += 1024) {
        const uint32_t s = c + tid;
        uint32_t size = 0, lo = 0;
        if (s < num_segments) {
            lo = off[s];
            size = off[s + 1] - lo;
        }
        const bool large = size > small_max;
        const uint32_t ntiles = large ? (size + tile - 1) / tile : 0u;
        if (s < num_segments && !large && size >= 2)
            small_list[atomicAdd(&ctrl->small_count, 1u)] = s;
        // Block-wide exclusive scans of (tiles, large flag), packed as two
        // 32-bit halves of one 64-bit sum.
        unsigned long long v = ((unsigned long long)ntiles << 32) | (large ? 1u : 0u);
        unsigned long long x = v;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ unsigned long long s_w64[32];
        if (lane == 31) s_w64[warp] = x;
        __syncthreads();
        unsigned long long off64 = 0;
        for (uint32_t w = 0; w < warp; ++w) off64 += s_w64[w];
        const unsigned long long excl = off64 + x - v;
        const uint32_t t0 = s_carry[0] + (uint32_t)(excl >> 32);
        const uint32_t ordinal = s_carry[1] + (uint32_t)(excl & 0xffffffffu);
        if (large) {
            large_first[ordinal] = lo;
            for (uint32_t k = 0; k < ntiles; ++k) {
                const uint32_t left = size - k * tile;
                tile_geo[t0 + k] = make_uint4(lo + k * tile, left < tile ? left : tile, t0, ordinal);
            }
        }
        __syncthreads();
        if (tid == 1023) {
            s_carry[0] = t0 + ntiles;
            s_carry[1] = ordinal + (large ? 1u : 0u);
        }
        __syncthreads();
    }
    if (tid == 0) {
        ctrl->seg_tiles = s_carry[0];
        ctrl->large_count = s_carry[1];
    }
}

// ---------------------------------------------------------------------------
// k_seg_hist: digit histograms of every large segment, added into
// hist[ordinal][4][256] (zeroed by the caller).  CTA c takes a contiguous run
// of tiles, so consecutive tiles mostly share a segment: counts accumulate in
// shared memory and are added to global memory only when the segment changes.
// Also clears the first scatter pass's status array.
// ---------------------------------------------------------------------------
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_seg_hist(const uint32_t* __restrict__ keys, const Ctrl* __restrict__ ctrl,
           const uint4* __restrict__ tile_geo, uint32_t* __restrict__ hist,
           uint4* __restrict__ clear, uint32_t clear_vec4) {
    __shared__ uint32_t s_h[PASSES * RADIX];
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = blockIdx.x * THREADS + tid; i < clear_vec4; i += gridDim.x * THREADS)
        clear[i] = make_uint4(0, 0, 0, 0);
    if (ctrl->err != 0) return;
    const uint32_t tiles = ctrl->seg_tiles;
    const uint32_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const uint32_t t_lo = blockIdx.x * per;
    const uint32_t t_hi = t_lo + per < tiles ? t_lo + per : tiles;
    for (uint32_t i = tid; i < PASSES * RADIX; i += THREADS) s_h[i] = 0;
    __syncthreads();
    uint32_t cur = 0xffffffffu;
    for (uint32_t t = t_lo; t < t_hi; ++t) {
        const uint4 g = tile_geo[t];
        if (g.w != cur) {
            if (cur != 0xffffffffu) {
                __syncthreads();
                for (uint32_t i = tid; i < PASSES * RADIX; i += THREADS) {
                    const uint32_t c = s_h[i];
                    if (c) atomicAdd(hist + (size_t)cur * PASSES * RADIX + i, c);
                    s_h[i] = 0;
                }
                __syncthreads();
            }
            cur = g.w;
        }
        for (uint32_t i = tid; i < g.y; i += THREADS) {
            const uint32_t k = ld_stream(keys + g.x + i);
#pragma unroll
            for (uint32_t p = 0; p < PASSES; ++p)
                atomicAdd(&s_h[p * RADIX + ((k >> (p * RADIX_BITS)) & (RADIX - 1))], 1u);
        }
    }
    __syncthreads();
    if (cur != 0xffffffffu)
        for (uint32_t i = tid; i < PASSES * RADIX; i += THREADS) {
            const uint32_t c = s_h[i];
            if (c) atomicAdd(hist + (size_t)cur * PASSES * RADIX + i, c);
        }
}

// ---------------------------------------------------------------------------
// k_seg_scan: per large segment (one CTA of 1024 threads = 4 digits x 256
// buckets), the exclusive prefix over buckets plus the segment's first item:
// the absolute first output slot of every bucket, written over the histogram.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_seg_scan(const Ctrl* __restrict__ ctrl, uint32_t* __restrict__ hist,
           const uint32_t* __restrict__ large_first) {
    __shared__ uint32_t s_warp[32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t p = tid >> 8;
    if (ctrl->err != 0) return;
    const uint32_t large = ctrl->large_count;
    for (uint32_t g = blockIdx.x; g < large; g += gridDim.x) {
        uint32_t* h = hist + (size_t)g * PASSES * RADIX;
        const uint32_t v = h[tid];
        uint32_t x = v;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t offv = 0;
        for (uint32_t w = p * (RADIX / 32); w < warp; ++w) offv += s_warp[w];
        h[tid] = large_first[g] + offv + x - v;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_small_sort: one CTA sorts a whole segment of at most CAP = THREADS *
// ITEMS items in shared memory: four stable counting-sort passes (Sec. 3)
// between two shared buffers, one read and one write of global memory.
// Segments come from small_list (count in ctrl->small_count); with
// off == nullptr the CTA sorts the single segment [0, single_n).
// Per pass: per-warp digit counts, their prefix over (digit, warp), then every
// warp ranks its items slot by slot (peers from one ballot per digit bit,
// positions from the warp's counters) and moves them to the other buffer.  A
// pass whose digit is the same for the whole segment is skipped.
// ---------------------------------------------------------------------------
template <int THREADS, int ITEMS, bool PAIRS>
__global__ void __launch_bounds__(THREADS)
k_small_sort(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
             const uint32_t* __restrict__ off, const uint32_t* __restrict__ small_list,
             const Ctrl* __restrict__ ctrl, uint32_t single_n) {
    constexpr uint32_t WARPS = THREADS / 32;
    constexpr uint32_t CAP = THREADS * ITEMS;
    constexpr uint32_t WARP_ITEMS = 32 * ITEMS;
    static_assert(THREADS >= (int)RADIX, "one thread per digit");
    extern __shared__ uint4 s_dyn[];
    uint32_t* const s_k = reinterpret_cast<uint32_t*>(s_dyn);  // [2][CAP]
    uint32_t* const s_v = s_k + 2 * CAP;                       // [2][CAP] (pairs)
    uint32_t* const s_w = s_v + (PAIRS ? 2 * CAP : 0);         // [WARPS][RADIX]
    __shared__ uint32_t s_scan[RADIX / 32];
    __shared__ uint32_t s_trivial;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t wofs = warp * WARP_ITEMS;

    uint32_t count = 1;
    if (off != nullptr) {
        if (ctrl->err != 0) return;
        count = ctrl->small_count;
    }
    for (uint32_t w = tid; w < WARPS * RADIX; w += THREADS) s_w[w] = 0;
    for (uint32_t idx = blockIdx.x; idx < count; idx += gridDim.x) {
        uint32_t lo = 0, m = single_n;
        if (off != nullptr) {
            const uint32_t s = small_list[idx];
            lo = off[s];
            m = off[s + 1] - lo;
        }
        for (uint32_t i = tid; i < m; i += THREADS) {
            s_k[i] = keys[lo + i];
            if (PAIRS) s_v[i] = vals[lo + i];
        }
        __syncthreads();
        uint32_t cur = 0;
        for (uint32_t p = 0; p < PASSES; ++p) {
            const uint32_t shift = p * RADIX_BITS;
            const uint32_t* ck = s_k + cur * CAP;
            uint32_t* row = s_w + warp * RADIX;
            const uint32_t left = m > wofs ? m - wofs : 0u;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (j * 32 + lane < left) atomicAdd(&row[(ck[wofs + j * 32 + lane] >> shift) & (RADIX - 1)], 1u);
            if (tid == 0) s_trivial = 0;
            __syncthreads();
            uint32_t c = 0;
            if (tid < RADIX) {
#pragma unroll
                for (uint32_t w = 0; w < WARPS; ++w) c += s_w[w * RADIX + tid];
                if (c == m) s_trivial = 1;
            }
            uint32_t x = c;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (tid < RADIX && lane == 31) s_scan[warp] = x;
            __syncthreads();
            if (s_trivial) {  // every item has the same digit: the pass is the identity
                for (uint32_t w = tid; w < WARPS * RADIX; w += THREADS) s_w[w] = 0;
                __syncthreads();
                continue;
            }
            if (tid < RADIX) {
                uint32_t offv = 0;
                for (uint32_t w = 0; w < warp; ++w) offv += s_scan[w];
                uint32_t run = offv + x - c;
#pragma unroll
                for (uint32_t w = 0; w < WARPS; ++w) {
                    const uint32_t t = s_w[w * RADIX + tid];
                    s_w[w * RADIX + tid] = run;
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
                const uint32_t d = (k >> shift) & (RADIX - 1);
                const uint32_t peers = match_label<RADIX_BITS>(d) & live;
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
            for (uint32_t i = lane; i < RADIX; i += 32) row[i] = 0;
            __syncthreads();
            cur ^= 1;
        }
        const uint32_t* fk = s_k + cur * CAP;
        const uint32_t* fv = s_v + cur * CAP;
        for (uint32_t i = tid; i < m; i += THREADS) {
            keys[lo + i] = fk[i];
            if (PAIRS) vals[lo + i] = fv[i];
        }
        __syncthreads();
    }
}

}  // namespace rs
