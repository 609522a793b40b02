// rs_segmented.cuh -- kernels of the segmented sort.
//
// A segmented sort sorts every segment [off[s], off[s+1]) of one array on its
// own (the paper has no segmented case; this is the plain definition applied
// per segment).  Segments are routed by size (rs_small.cuh has the first two):
//   tiny (2 <= size <= warp_max): k_warp_sort, one warp per segment, the whole
//       segment in that warp's shared memory for every pass;
//   small (warp_max < size <= small_max): k_small_sort, one CTA per segment,
//       the whole segment in shared memory -- one read and one write of every
//       item either way;
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
//  - Tiny segments are listed in tiny_list, small ones in small_list (order
//    irrelevant).
//  - The pass plan runs all four passes (caller -> alternate -> ... -> caller).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_seg_plan(const uint32_t* __restrict__ off, uint32_t num_segments, uint32_t n, uint32_t tile,
           uint32_t warp_max, uint32_t small_max, Ctrl* __restrict__ ctrl,
           uint32_t* __restrict__ sticky, uint4* __restrict__ tile_geo,
           uint32_t* __restrict__ tiny_list, uint32_t* __restrict__ small_list,
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
        if (s < num_segments && !large && size >= 2) {
            if (size <= warp_max)
                tiny_list[atomicAdd(&ctrl->tiny_count, 1u)] = s;
            else
                small_list[atomicAdd(&ctrl->small_count, 1u)] = s;
        }
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
           uint4* __restrict__ clear, uint32_t clear_vec4, uint32_t key_type) {
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
            const uint32_t k = key_to_ordered(ld_stream(keys + g.x + i), key_type);
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

}  // namespace rs
