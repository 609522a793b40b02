// rs_segmented_wide.cuh -- kernels of the segmented sort of wide items
// (64-bit keys, or 32-bit keys carrying 64-bit values): the one-warp sort of
// short segments and the per-segment digit histograms of 64-bit keys.  The
// large segments take the scatter passes (k_onesweep<..., SEG>) with the
// items' widths, as the 32-bit segmented sort does.
#pragma once

#include "rs_device.cuh"

namespace rs {

constexpr int WIDE_WARP_THREADS = 256;  // 8 independent warps per CTA

// Bytes of one warp's region of k_warp_sort_wide: keys [2][32 * ITEMS],
// values [2][32 * ITEMS] (key-value sorts), digit counters [256].
template <typename K, typename V, bool PAIRS, int ITEMS>
struct WideWarpSmem {
    static constexpr uint32_t CAP = 32 * ITEMS;
    static constexpr size_t KEYS = 2 * CAP * sizeof(K);
    static constexpr size_t VALS = PAIRS ? 2 * CAP * sizeof(V) : 0;
    static constexpr size_t PER_WARP = KEYS + VALS + RADIX * sizeof(uint32_t);
    static constexpr size_t BYTES = (WIDE_WARP_THREADS / 32) * PER_WARP;
    static_assert(KEYS % 16 == 0 && VALS % 16 == 0, "8-byte items stay aligned");
};

// ---------------------------------------------------------------------------
// k_warp_sort_wide: every warp sorts whole segments of at most 32 * ITEMS
// items (those in `list`, count ctrl->tiny_count), one at a time, in its own
// shared-memory region: one stable counting-sort pass (Sec. 3) per 8-bit
// digit of the key between two shared buffers -- the digit counts (shared
// atomics), their exclusive prefix, then the items slot by slot in input
// order (peers from one ballot per digit bit, the lowest advancing the
// digit's counter by the group's size).  A pass whose digit is the same for
// the whole segment is skipped.  Typed keys are mapped onto their ordered
// words when read and back when written.
// ---------------------------------------------------------------------------
template <typename K, typename V, bool PAIRS, int ITEMS>
__global__ void __launch_bounds__(WIDE_WARP_THREADS)
k_warp_sort_wide(K* __restrict__ keys, V* __restrict__ vals, const uint32_t* __restrict__ off,
                 const uint32_t* __restrict__ list, const Ctrl* __restrict__ ctrl,
                 uint32_t key_type) {
    using L = WideWarpSmem<K, V, PAIRS, ITEMS>;
    constexpr uint32_t CAP = L::CAP;
    constexpr uint32_t NPASS = sizeof(K);  // one 8-bit digit per key byte
    constexpr uint32_t WARPS = WIDE_WARP_THREADS / 32;
    constexpr uint32_t PL = RADIX / 32;    // counters scanned per lane
    extern __shared__ uint4 s_dyn[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    char* const base = reinterpret_cast<char*>(s_dyn) + warp * L::PER_WARP;
    K* const s_k = reinterpret_cast<K*>(base);
    V* const s_v = reinterpret_cast<V*>(base + L::KEYS);
    uint32_t* const cnt = reinterpret_cast<uint32_t*>(base + L::KEYS + L::VALS);
    const uint32_t lt = lanemask_lt();
    if (ctrl->err != 0) return;
    const uint32_t count = ctrl->tiny_count;
    for (uint32_t idx = blockIdx.x * WARPS + warp; idx < count; idx += gridDim.x * WARPS) {
        const uint32_t s = list[idx];
        const uint32_t lo = off[s], m = off[s + 1] - lo;
        for (uint32_t i = lane; i < m; i += 32) {
            s_k[i] = key_to_ordered(keys[lo + i], key_type);
            if (PAIRS) s_v[i] = vals[lo + i];
        }
        uint32_t cur = 0;
        for (uint32_t p = 0; p < NPASS; ++p) {
            auto digit = [p](K k) { return (uint32_t)(k >> (8u * p)) & (RADIX - 1); };
            for (uint32_t b = lane; b < RADIX; b += 32) cnt[b] = 0;
            __syncwarp();
            const K* ck = s_k + cur * CAP;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((uint32_t)j * 32 >= m) break;  // warp-uniform
                const uint32_t i = j * 32 + lane;
                if (i < m) atomicAdd(&cnt[digit(ck[i])], 1u);
            }
            __syncwarp();
            uint32_t c[PL];
            uint32_t tot = 0;
            bool trivial = false;
#pragma unroll
            for (uint32_t q = 0; q < PL; ++q) {
                c[q] = cnt[lane * PL + q];
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
                cnt[lane * PL + q] = run;
                run += c[q];
            }
            __syncwarp();
            K* nk = s_k + (cur ^ 1) * CAP;
            const V* cv = s_v + cur * CAP;
            V* nv = s_v + (cur ^ 1) * CAP;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((uint32_t)j * 32 >= m) break;  // warp-uniform
                const uint32_t i = j * 32 + lane;
                const uint32_t live = prefix_lanes(j * 32, m);
                const K k = i < m ? ck[i] : K(0);
                const uint32_t d = digit(k);
                const uint32_t peers = match_label<RADIX_BITS>(d) & live;
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
        const K* fk = s_k + cur * CAP;
        const V* fv = s_v + cur * CAP;
        for (uint32_t i = lane; i < m; i += 32) {
            keys[lo + i] = key_from_ordered(fk[i], key_type);
            if (PAIRS) vals[lo + i] = fv[i];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// k_seg_hist64: the eight digit histograms of every large segment of 64-bit
// keys, added into hist[ordinal][8][256] (zeroed by the caller).  One CTA
// per SM takes a contiguous run of tiles (consecutive tiles mostly share a
// segment), counts into a CTA-private shared histogram with shared atomics,
// and adds it to the segment's global histogram when the segment changes.
// Also clears the first scatter pass's status array.  TYPED: keys are mapped
// onto their ordered words first.
// ---------------------------------------------------------------------------
constexpr uint32_t SEG_HIST64_THREADS = 1024;

template <bool TYPED>
__global__ void __launch_bounds__(SEG_HIST64_THREADS, 1)
k_seg_hist64(const unsigned long long* __restrict__ keys, const Ctrl* __restrict__ ctrl,
             const uint4* __restrict__ tile_geo, uint32_t* __restrict__ hist,
             uint4* __restrict__ clear, uint32_t clear_vec4, uint32_t key_type) {
    __shared__ uint32_t s_h[PASSES64 * RADIX];
    constexpr uint32_t T = SEG_HIST64_THREADS;
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = blockIdx.x * T + tid; i < clear_vec4; i += gridDim.x * T)
        clear[i] = make_uint4(0, 0, 0, 0);
    if (ctrl->err != 0) return;
    const uint32_t tiles = ctrl->seg_tiles;
    const uint32_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const uint32_t t_lo = blockIdx.x * per;
    const uint32_t t_hi = t_lo + per < tiles ? t_lo + per : tiles;
    if (t_lo >= t_hi) return;
    for (uint32_t i = tid; i < PASSES64 * RADIX; i += T) s_h[i] = 0;
    __syncthreads();
    auto flush = [&](uint32_t seg) {
        __syncthreads();
        for (uint32_t bin = tid; bin < PASSES64 * RADIX; bin += T) {
            const uint32_t c = s_h[bin];
            if (c) atomicAdd(hist + (size_t)seg * PASSES64 * RADIX + bin, c);
            s_h[bin] = 0;
        }
        __syncthreads();
    };
    uint32_t cur = 0xffffffffu;
    for (uint32_t t = t_lo; t < t_hi; ++t) {
        const uint4 g = tile_geo[t];  // the same for every thread of the CTA
        if (g.w != cur) {
            if (cur != 0xffffffffu) flush(cur);
            cur = g.w;
        }
        for (uint32_t i = tid; i < g.y; i += T) {
            unsigned long long k = __ldcs(keys + g.x + i);
            if (TYPED) k = key_to_ordered(k, key_type);
#pragma unroll
            for (uint32_t p = 0; p < PASSES64; ++p)
                atomicAdd(&s_h[p * RADIX + ((uint32_t)(k >> (8u * p)) & (RADIX - 1))], 1u);
        }
    }
    flush(cur);
}

}  // namespace rs
