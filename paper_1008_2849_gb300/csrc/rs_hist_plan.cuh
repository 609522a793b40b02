// rs_hist_plan.cuh -- the two small kernels that precede the scatter passes:
//   k_hist4  one read of the keys builds all four digit histograms (the
//            counting step of Sec. 3, for every digit at once);
//   k_plan   exclusive prefix over the buckets of every digit (Sec. 3 "prefix
//            sum"; Alg. 2 PrefixSum) and the pass plan.
#pragma once

#include "rs_device.cuh"

namespace rs {

// ---------------------------------------------------------------------------
// k_hist4: H[p][b] for p = 0..3 in one pass over the keys, added into
// hist[p * 256 + b] (which the caller zeroes).
//
// Keys are read as 16-byte vectors (a scalar head and tail handle a base that
// is only 4-byte aligned) into a CTA-private shared histogram, which is added
// to the global one at the end.  How a warp updates the shared histogram is
// a tuning choice (MODE):
//   HIST_ATOMIC   every lane adds 1 to its bin;
//   HIST_LEADER   lanes whose digit equals lane 0's are added as one group
//                 (cheap, and it removes the worst shared-memory serialisation
//                 when most keys share a digit), the others add 1 each;
//   HIST_MATCH    lanes are grouped by digit with one ballot per digit bit and
//                 the lowest lane of every group adds the group's size.
// The kernel also clears the look-back status array of the first scatter
// pass.
// ---------------------------------------------------------------------------
constexpr int HIST_ATOMIC = 0;
constexpr int HIST_LEADER = 1;
constexpr int HIST_MATCH = 2;
constexpr int HIST_COLUMNS = 3;  // k_hist4_cols

// TYPED: keys are mapped onto their ordered words (key_type) before counting;
// unsigned keys use the instances without the map.
template <int THREADS, int MODE, bool TYPED>
__global__ void __launch_bounds__(THREADS)
k_hist4(const uint32_t* __restrict__ keys, uint32_t n, uint32_t* __restrict__ hist,
        uint4* __restrict__ clear, uint32_t clear_vec4, uint32_t key_type) {
    __shared__ uint32_t s_h[PASSES * RADIX];
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31;
    for (uint32_t i = tid; i < PASSES * RADIX; i += THREADS) s_h[i] = 0;

    const uint32_t gtid = blockIdx.x * THREADS + tid;
    const uint32_t gsize = gridDim.x * THREADS;
    for (uint32_t i = gtid; i < clear_vec4; i += gsize) clear[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    uint32_t head = (uint32_t)(((16u - ((uintptr_t)keys & 15u)) & 15u) >> 2);
    if (head > n) head = n;
    const uint32_t body4 = (n - head) >> 2;
    const uint32_t tail = head + body4 * 4;
    const uint4* __restrict__ body = reinterpret_cast<const uint4*>(keys + head);

    auto count_key = [&](uint32_t key, bool ok) {
        if (TYPED) key = key_to_ordered(key, key_type);
#pragma unroll
        for (uint32_t p = 0; p < PASSES; ++p) {
            const uint32_t d = (key >> (p * RADIX_BITS)) & (RADIX - 1);
            uint32_t* bin = &s_h[p * RADIX + d];
            if (MODE == HIST_ATOMIC) {
                if (ok) atomicAdd(bin, 1u);
            } else if (MODE == HIST_LEADER) {
                const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
                const uint32_t same = __ballot_sync(0xffffffffu, ok && d == d0);
                if (ok) {
                    if (d != d0) atomicAdd(bin, 1u);
                    else if (lane == (uint32_t)(__ffs(same) - 1)) atomicAdd(bin, (uint32_t)__popc(same));
                }
            } else {
                const uint32_t peers = match_label<RADIX_BITS>(d) & __ballot_sync(0xffffffffu, ok);
                if (ok && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(bin, (uint32_t)__popc(peers));
            }
        }
    };

    // Warp-uniform loop: every iteration a warp takes 2 x 32 consecutive
    // vectors, so all 32 lanes always take part in the warp votes.
    const uint32_t gwarp = gtid >> 5;
    const uint32_t nwarps = gsize >> 5;
    for (uint32_t c = gwarp * 64; c < body4; c += nwarps * 64) {
        const uint32_t i0 = c + lane, i1 = c + 32 + lane;
        const bool ok0 = i0 < body4, ok1 = i1 < body4;
        const uint4 v0 = ok0 ? ld_stream(body + i0) : make_uint4(0, 0, 0, 0);
        const uint4 v1 = ok1 ? ld_stream(body + i1) : make_uint4(0, 0, 0, 0);
        count_key(v0.x, ok0); count_key(v0.y, ok0); count_key(v0.z, ok0); count_key(v0.w, ok0);
        count_key(v1.x, ok1); count_key(v1.y, ok1); count_key(v1.z, ok1); count_key(v1.w, ok1);
    }
    // At most 3 keys before the first 16-byte boundary and 3 after the last.
    if (blockIdx.x == 0 && tid < 8) {
        const uint32_t i = tid < 4 ? tid : tail + (tid - 4);
        const bool ok = tid < 4 ? i < head : i < n;
        if (ok) {
            const uint32_t key = TYPED ? key_to_ordered(keys[i], key_type) : keys[i];
#pragma unroll
            for (uint32_t p = 0; p < PASSES; ++p)
                atomicAdd(&s_h[p * RADIX + ((key >> (p * RADIX_BITS)) & (RADIX - 1))], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < PASSES * RADIX; i += THREADS) {
        const uint32_t c = s_h[i];
        if (c) atomicAdd(hist + i, c);
    }
}

// ---------------------------------------------------------------------------
// k_hist4_cols: the same histograms with one private column per lane: bin b
// of digit p, as seen by lane l, lives at word (p*256 + b)*32 + l of a
// 128 KiB shared array, so the 32 lanes of a warp always add into 32
// different banks (one shared-memory wavefront per warp-wide add, whatever
// the keys).  Columns are summed (in rotated order, again conflict-free) at
// the end.  One CTA per SM.
// ---------------------------------------------------------------------------
constexpr uint32_t HIST_COL_WORDS = PASSES * RADIX * 32;

template <int THREADS, bool TYPED>
__global__ void __launch_bounds__(THREADS, 1)
k_hist4_cols(const uint32_t* __restrict__ keys, uint32_t n, uint32_t* __restrict__ hist,
             uint4* __restrict__ clear, uint32_t clear_vec4, uint32_t key_type) {
    extern __shared__ uint4 s_cols4[];
    uint32_t* const s_col = reinterpret_cast<uint32_t*>(s_cols4);
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31;
    pdl_launch_next();  // the plan kernel may launch; it waits for this one
    for (uint32_t i = tid; i < HIST_COL_WORDS / 4; i += THREADS) s_cols4[i] = make_uint4(0, 0, 0, 0);
    const uint32_t gtid = blockIdx.x * THREADS + tid;
    const uint32_t gsize = gridDim.x * THREADS;
    for (uint32_t i = gtid; i < clear_vec4; i += gsize) clear[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    uint32_t head = (uint32_t)(((16u - ((uintptr_t)keys & 15u)) & 15u) >> 2);
    if (head > n) head = n;
    const uint32_t body4 = (n - head) >> 2;
    const uint32_t tail = head + body4 * 4;
    const uint4* __restrict__ body = reinterpret_cast<const uint4*>(keys + head);
    uint32_t* const mycol = s_col + lane;
    auto count_key = [&](uint32_t key) {
        if (TYPED) key = key_to_ordered(key, key_type);
#pragma unroll
        for (uint32_t p = 0; p < PASSES; ++p)
            atomicAdd(mycol + ((p * RADIX + ((key >> (p * RADIX_BITS)) & (RADIX - 1))) << 5), 1u);
    };
    // HIST_LOADS independent 16-byte loads in flight per thread and
    // iteration (64 KiB per SM): enough bytes in flight to cover the HBM
    // latency at full bandwidth.
    constexpr uint32_t HIST_LOADS = 4;
    for (uint32_t i = gtid; i < body4; i += HIST_LOADS * gsize) {
        uint4 v[HIST_LOADS];
#pragma unroll
        for (uint32_t u = 0; u < HIST_LOADS; ++u)
            v[u] = i + u * gsize < body4 ? ld_stream(body + i + u * gsize) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (uint32_t u = 0; u < HIST_LOADS; ++u) {
            if (i + u * gsize < body4) {
                count_key(v[u].x);
                count_key(v[u].y);
                count_key(v[u].z);
                count_key(v[u].w);
            }
        }
    }
    if (blockIdx.x == 0 && tid < 8) {
        const uint32_t i = tid < 4 ? tid : tail + (tid - 4);
        const bool ok = tid < 4 ? i < head : i < n;
        if (ok) count_key(keys[i]);
    }
    __syncthreads();
    for (uint32_t bin = tid; bin < PASSES * RADIX; bin += THREADS) {
        uint32_t c = 0;
#pragma unroll 8
        for (uint32_t j = 0; j < 32; ++j) c += s_col[(bin << 5) + ((j + bin) & 31)];
        if (c) atomicAdd(hist + bin, c);
    }
}

// ---------------------------------------------------------------------------
// k_plan: G[p][b] = sum_{b' < b} H[p][b'] and the pass plan.  One CTA of
// 1024 threads, thread (p, b) = (tid / 256, tid % 256).
//
// A pass whose digit takes one value for every key is the identity (a stable
// partition into one bucket).  Such passes are skipped, except that the
// number of executed passes is kept even (one trivial pass is run if needed)
// so that the ping-pong between the caller's arrays and the alternate
// buffers ends in the caller's arrays.
//
// MSD-first order (Alg. 2, "reverse sorting"), when msd_allowed: if digit 3
// is not trivial and no digit-3 bucket holds more than bucket_cap keys, the
// plan runs one pass by digit 3 (plan slot MSD_SLOT, caller's arrays ->
// alternate buffers) and skips passes 0..3; every bucket is then sorted on
// chip from the alternate buffers back into the caller's arrays (its digit 3
// is constant, so that pass is trivial there).  msd_off[b] is bucket b's
// first slot (msd_off[256] = n); non-empty buckets of at most warp_max keys
// are listed in tiny_list (one-warp sort), larger ones in small_list
// (one-CTA sort).
// ---------------------------------------------------------------------------
template <int NPASS>
__global__ void __launch_bounds__(1024)
k_plan(Ctrl* __restrict__ ctrl, uint32_t n, uint32_t msd_allowed, uint32_t warp_max,
       uint32_t bucket_cap, uint32_t* __restrict__ msd_off, uint32_t* __restrict__ tiny_list,
       uint32_t* __restrict__ small_list) {
    static_assert(NPASS == 4 || NPASS == 8, "32-bit or 64-bit keys");
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_trivial[NPASS];
    __shared__ uint32_t s_big;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t b = tid & (RADIX - 1);
    pdl_launch_next();
    pdl_wait();  // the histograms are complete
    if (tid < NPASS) s_trivial[tid] = 0;
    if (tid == 0) s_big = 0;
    // Thread (p, b): p = tid / 256 (+ 4 in the second round for 64-bit keys).
    uint32_t h3 = 0, first3 = 0;  // digit 3, for the MSD-first order
    for (uint32_t round = 0; round < NPASS / 4; ++round) {
        const uint32_t p = (tid >> 8) + 4 * round;
        const uint32_t h = ctrl->hist[p][b];
        uint32_t x = h;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t off = 0;
        for (uint32_t w = (tid >> 8) * (RADIX / 32); w < warp; ++w) off += s_warp[w];
        const uint32_t first = off + x - h;
        ctrl->gofs[p][b] = first;
        if (h == n) s_trivial[p] = 1;
        if (p == PASSES - 1) {
            h3 = h;
            first3 = first;
            if (h > bucket_cap) s_big = 1;
        }
        __syncthreads();  // s_warp is reused by the next round
    }
    const bool msd = NPASS == 4 && msd_allowed && !s_trivial[PASSES - 1] && !s_big;
    if (msd && (tid >> 8) == PASSES - 1) {
        msd_off[b] = first3;
        if (b == RADIX - 1) msd_off[RADIX] = n;
        if (h3 > 0) {
            if (h3 <= warp_max)
                tiny_list[atomicAdd(&ctrl->tiny_count, 1u)] = b;
            else
                small_list[atomicAdd(&ctrl->small_count, 1u)] = b;
        }
    }
    if (tid == 0 && msd) {
        for (uint32_t q = 0; q < PASSES; ++q) ctrl->dir[q] = DIR_SKIP;
        ctrl->dir[MSD_SLOT] = DIR_A_TO_B;
    } else if (tid == 0) {
        ctrl->dir[MSD_SLOT] = DIR_SKIP;
        uint32_t trivial[NPASS], executed = 0;
        for (uint32_t q = 0; q < NPASS; ++q) {
            trivial[q] = s_trivial[q];
            executed += trivial[q] ? 0 : 1;
        }
        if (executed & 1) {
            for (uint32_t q = 0; q < NPASS; ++q)
                if (trivial[q]) { trivial[q] = 0; break; }
        }
        uint32_t parity = 0;
        for (uint32_t q = 0; q < NPASS; ++q) {
            if (trivial[q]) {
                ctrl->dir[q] = DIR_SKIP;
            } else {
                ctrl->dir[q] = parity ? DIR_B_TO_A : DIR_A_TO_B;
                parity ^= 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_msd_plan: the plan of one stable counting-sort pass by the most
// significant digit (digit 3; Alg. 2's local MSD pass): G[3][b] = the
// exclusive prefix of H[3], copied to bucket_off[0..255] with
// bucket_off[256] = n, and the pass run (plan slot MSD_SLOT) from the input
// to the output arrays even when every key has the same digit (then it is a
// copy).  One CTA of 256 threads, thread b = bucket b.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(RADIX)
k_msd_plan(Ctrl* __restrict__ ctrl, uint32_t n, uint32_t* __restrict__ bucket_off) {
    __shared__ uint32_t s_warp[RADIX / 32];
    const uint32_t b = threadIdx.x, lane = b & 31, warp = b >> 5;
    const uint32_t h = ctrl->hist[PASSES - 1][b];
    uint32_t x = h;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t off = 0;
    for (uint32_t w = 0; w < warp; ++w) off += s_warp[w];
    const uint32_t first = off + x - h;
    ctrl->gofs[PASSES - 1][b] = first;
    bucket_off[b] = first;
    if (b == 0) {
        bucket_off[RADIX] = n;
        ctrl->dir[MSD_SLOT] = DIR_A_TO_B;
    }
}

// ---------------------------------------------------------------------------
// k_hist8: the eight digit histograms of 64-bit keys (K = 64, D = 8) in one
// read of the keys, added into hist[p * 256 + b] (zeroed by the caller), via
// a CTA-private shared histogram.  Typed keys (TYPED) are counted by the
// digits of their ordered words.  Also clears the first pass's status array.
// ---------------------------------------------------------------------------
template <int THREADS, bool TYPED>
__global__ void __launch_bounds__(THREADS)
k_hist8(const unsigned long long* __restrict__ keys, uint32_t n, uint32_t* __restrict__ hist,
        uint4* __restrict__ clear, uint32_t clear_vec4, uint32_t key_type) {
    __shared__ uint32_t s_h[PASSES64 * RADIX];
    const uint32_t tid = threadIdx.x;
    pdl_launch_next();  // the plan kernel may launch; it waits for this one
    for (uint32_t i = tid; i < PASSES64 * RADIX; i += THREADS) s_h[i] = 0;
    const uint32_t gtid = blockIdx.x * THREADS + tid;
    const uint32_t gsize = gridDim.x * THREADS;
    for (uint32_t i = gtid; i < clear_vec4; i += gsize) clear[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (uint32_t i = gtid; i < n; i += gsize) {
        unsigned long long k = __ldcs(keys + i);
        if (TYPED) k = key_to_ordered(k, key_type);
        const uint32_t lo = (uint32_t)k, hi = (uint32_t)(k >> 32);
#pragma unroll
        for (uint32_t p = 0; p < 4; ++p) {
            atomicAdd(&s_h[p * RADIX + ((lo >> (8 * p)) & (RADIX - 1))], 1u);
            atomicAdd(&s_h[(p + 4) * RADIX + ((hi >> (8 * p)) & (RADIX - 1))], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < PASSES64 * RADIX; i += THREADS) {
        const uint32_t c = s_h[i];
        if (c) atomicAdd(hist + i, c);
    }
}

}  // namespace rs
