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
//  - The pass plan runs all npass passes (four, or eight for 64-bit keys;
//    caller -> alternate -> ... -> caller).
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024)
k_seg_plan(const uint32_t* __restrict__ off, uint32_t num_segments, uint32_t n, uint32_t tile,
           uint32_t warp_max, uint32_t small_max, Ctrl* __restrict__ ctrl,
           uint32_t* __restrict__ sticky, uint4* __restrict__ tile_geo,
           uint32_t* __restrict__ tiny_list, uint32_t* __restrict__ small_list,
           uint32_t* __restrict__ large_first /* [S] first item of large ordinal */,
           uint32_t npass = PASSES) {
    __shared__ uint32_t s_carry[2];  // tiles and large segments before this chunk
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_launch_next();
    pdl_wait();

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
        for (uint32_t p = 0; p < npass; ++p) ctrl->dir[p] = (p & 1) ? DIR_B_TO_A : DIR_A_TO_B;
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
// hist[ordinal][4][256] (zeroed by the caller).  One CTA of 1024 threads per
// SM takes a contiguous run of tiles, so consecutive tiles mostly share a
// segment.  Counts accumulate in per-lane shared-memory columns (bin b of
// digit p as seen by lane l at word (p*256 + b)*32 + l: the 32 lanes of a warp
// always add into 32 different banks) and are summed into global memory only
// when the segment changes.  Also clears the first scatter pass's status
// array.  TYPED: keys are mapped onto their ordered words first.
// ---------------------------------------------------------------------------
constexpr uint32_t SEG_HIST_THREADS = 1024;
constexpr uint32_t SEG_HIST_COL_WORDS = PASSES * RADIX * 32;
constexpr uint32_t SEG_HIST_GEO_CHUNK = 1024;  // tile geometries staged at a time

template <bool TYPED>
__global__ void __launch_bounds__(SEG_HIST_THREADS, 1)
k_seg_hist(const uint32_t* __restrict__ keys, const Ctrl* __restrict__ ctrl,
           const uint4* __restrict__ tile_geo, uint32_t* __restrict__ hist,
           uint4* __restrict__ clear, uint32_t clear_vec4, uint32_t key_type) {
    extern __shared__ uint4 s_cols4[];
    uint32_t* const s_col = reinterpret_cast<uint32_t*>(s_cols4);
    constexpr uint32_t T = SEG_HIST_THREADS;
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    pdl_launch_next();
    pdl_wait();  // the planner and the on-chip sorts are complete
    for (uint32_t i = blockIdx.x * T + tid; i < clear_vec4; i += gridDim.x * T)
        clear[i] = make_uint4(0, 0, 0, 0);
    if (ctrl->err != 0) return;
    const uint32_t tiles = ctrl->seg_tiles;
    const uint32_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const uint32_t t_lo = blockIdx.x * per;
    const uint32_t t_hi = t_lo + per < tiles ? t_lo + per : tiles;
    if (t_lo >= t_hi) return;
    for (uint32_t i = tid; i < SEG_HIST_COL_WORDS / 4; i += T) s_cols4[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t* const mycol = s_col + lane;
    auto count_key = [&](uint32_t k) {
        if (TYPED) k = key_to_ordered(k, key_type);
#pragma unroll
        for (uint32_t p = 0; p < PASSES; ++p)
            atomicAdd(mycol + ((p * RADIX + ((k >> (p * RADIX_BITS)) & (RADIX - 1))) << 5), 1u);
    };
    // Thread `bin` sums (and clears) the 32 columns of one bin, in rotated
    // order so that a warp's reads fall into 32 different banks.
    auto flush = [&](uint32_t seg) {
        __syncthreads();
        for (uint32_t bin = tid; bin < PASSES * RADIX; bin += T) {
            uint32_t c = 0;
#pragma unroll 8
            for (uint32_t j = 0; j < 32; ++j) {
                const uint32_t w = (bin << 5) + ((j + bin) & 31);
                c += s_col[w];
                s_col[w] = 0;
            }
            if (c) atomicAdd(hist + (size_t)seg * PASSES * RADIX + bin, c);
        }
        __syncthreads();
    };
    // Counts the keys [lo, hi): up to 3 before the first 16-byte boundary
    // and up to 3 after the last one one by one, the rest as 16-byte
    // vectors, two in flight per thread.
    auto count_range = [&](uint32_t lo, uint32_t hi) {
        const uint32_t* src = keys + lo;
        const uint32_t m = hi - lo;
        uint32_t head = (uint32_t)(((16u - ((uintptr_t)src & 15u)) & 15u) >> 2);
        if (head > m) head = m;
        const uint32_t nvec = (m - head) >> 2;
        const uint4* body = reinterpret_cast<const uint4*>(src + head);
        uint32_t v = tid;
        for (; v + T < nvec; v += 2 * T) {
            const uint4 x = ld_stream(body + v), y = ld_stream(body + v + T);
            count_key(x.x); count_key(x.y); count_key(x.z); count_key(x.w);
            count_key(y.x); count_key(y.y); count_key(y.z); count_key(y.w);
        }
        if (v < nvec) {
            const uint4 x = ld_stream(body + v);
            count_key(x.x); count_key(x.y); count_key(x.z); count_key(x.w);
        }
        const uint32_t tail = head + nvec * 4;
        if (tid < head) count_key(ld_stream(src + tid));
        if (tid < 4 && tail + tid < m) count_key(ld_stream(src + tail + tid));
    };
    // The CTA's tiles, a chunk of geometries at a time in shared memory.
    // Consecutive tiles of one segment cover consecutive keys, so every run
    // of them is counted as one range (no per-tile wait on its geometry).
    __shared__ uint4 s_g[SEG_HIST_GEO_CHUNK];
    uint32_t cur = 0xffffffffu;
    for (uint32_t c0 = t_lo; c0 < t_hi; c0 += SEG_HIST_GEO_CHUNK) {
        const uint32_t cn = t_hi - c0 < SEG_HIST_GEO_CHUNK ? t_hi - c0 : SEG_HIST_GEO_CHUNK;
        __syncthreads();  // the previous chunk is no longer read
        for (uint32_t i = tid; i < cn; i += T) s_g[i] = tile_geo[c0 + i];
        __syncthreads();
        for (uint32_t ra = 0; ra < cn;) {
            const uint32_t seg = s_g[ra].w;
            uint32_t rb = ra;
            while (rb + 1 < cn && s_g[rb + 1].w == seg) ++rb;
            if (seg != cur) {
                if (cur != 0xffffffffu) flush(cur);
                cur = seg;
            }
            count_range(s_g[ra].x, s_g[rb].x + s_g[rb].y);
            ra = rb + 1;
        }
    }
    flush(cur);
}

// ---------------------------------------------------------------------------
// k_seg_scan: per large segment (one CTA of 1024 threads = 4 digits x 256
// buckets, twice for the eight digits of 64-bit keys), the exclusive prefix
// over buckets plus the segment's first item: the absolute first output slot
// of every bucket, written over the histogram hist[segment][NP][256].
// ---------------------------------------------------------------------------
template <int NP = PASSES>
__global__ void __launch_bounds__(1024)
k_seg_scan(const Ctrl* __restrict__ ctrl, uint32_t* __restrict__ hist,
           const uint32_t* __restrict__ large_first) {
    static_assert(NP == 4 || NP == 8, "32-bit or 64-bit keys");
    __shared__ uint32_t s_warp[32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t p = tid >> 8;
    pdl_launch_next();
    pdl_wait();  // the segment histograms are complete
    if (ctrl->err != 0) return;
    const uint32_t large = ctrl->large_count;
    for (uint32_t g = blockIdx.x; g < large; g += gridDim.x)
    for (uint32_t round = 0; round < NP / 4; ++round) {
        uint32_t* h = hist + ((size_t)g * NP + 4 * round) * RADIX;
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
