// rs_onesweep.cuh -- k_onesweep, one stable counting-sort pass (Sec. 3/4)
// per launch: per-tile ranking with warp match-any, a decoupled look-back
// across tiles for the tile's share of every bucket, staging of the tile in
// shared memory in bucket order, and coalesced stores of every bucket run --
// the GPU counterpart of the software write-combining buffers of Sec. 2.
#pragma once

#include "rs_device.cuh"

namespace rs {

// ---------------------------------------------------------------------------
// k_onesweep: one stable counting-sort pass by digit `pass` over tiles of
// TILE = THREADS * ITEMS items.
//
// Layout of a tile in registers: warp w holds tile items [w*32*ITEMS,
// (w+1)*32*ITEMS); item j of lane l is tile item w*32*ITEMS + j*32 + l, so
// every load instruction of a warp reads 128 contiguous bytes, and the
// (warp, j, lane) order is the input order -- which is what keeps the
// ranking stable.
//
// Ranking: for every item, match-any gives the lanes of the warp holding the
// same digit; the lowest of them adds the group's size to the warp's
// counter of that digit; an item's rank is the counter's old value plus the
// number of its peers on lower lanes.  Warp counters are then turned into
// per-warp exclusive offsets and the tile's per-digit count c[b].
//
// Look-back: the tile publishes c[b] (flag AGG; the first tile publishes
// INC), then thread b walks back over the tiles before it, adding AGG counts
// until it meets an INC prefix, and publishes its own inclusive prefix
// (INC).  Tile ids come from an atomic counter, so every tile before this
// one belongs to a CTA that is already running and will publish.  Every wait
// is bounded by spin_limit polls; when it runs out the kernel records
// ERR_TIMEOUT and the CTA (and every CTA that sees the error) writes nothing.
//
// Scatter: keys are written to shared memory at their tile position (bucket
// order), then read back in slot order and stored to
//   dst[G[b] + prefix_before_this_tile[b] + (slot - tile_excl[b])],
// so consecutive threads store consecutive addresses of one bucket run.
// Values follow through the same staging buffer.  Every global store is
// checked against n (ERR_BOUNDS instead of a fault).
// ---------------------------------------------------------------------------
template <int THREADS, int ITEMS, bool PAIRS, typename S>
__global__ void __launch_bounds__(THREADS, (THREADS >= 512 ? 2 : 4))
k_onesweep(uint32_t* __restrict__ ka, uint32_t* __restrict__ va,
           uint32_t* __restrict__ kb, uint32_t* __restrict__ vb,
           uint32_t n, uint32_t pass, Ctrl* __restrict__ ctrl, uint32_t* __restrict__ sticky,
           S* __restrict__ status, S* __restrict__ status_clear,
           uint32_t spin_limit, uint32_t debug) {
    static_assert(THREADS >= (int)RADIX && THREADS % 32 == 0, "one thread per digit");
    using SW = StatusWord<S>;
    constexpr uint32_t WARPS = THREADS / 32;
    constexpr uint32_t TILE = THREADS * ITEMS;
    constexpr uint32_t WARP_ITEMS = 32 * ITEMS;

    __shared__ uint32_t s_wcnt[WARPS][RADIX + 1];  // bin RADIX: items past n
    __shared__ uint32_t s_excl[RADIX];
    __shared__ uint32_t s_gofs[RADIX];
    __shared__ uint32_t s_scan[RADIX / 32];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_abort;
    extern __shared__ uint32_t s_stage[];  // TILE words

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Clear this CTA's slot of the next pass's status array (its last user,
    // the previous pass, has completed).
    if (status_clear != nullptr)
        for (uint32_t b = tid; b < RADIX; b += THREADS)
            status_clear[(size_t)blockIdx.x * RADIX + b] = 0;

    const uint32_t dir = ctrl->dir[pass];
    if (dir == DIR_SKIP) return;
    const uint32_t* __restrict__ src_k = dir == DIR_A_TO_B ? ka : kb;
    uint32_t* __restrict__ dst_k = dir == DIR_A_TO_B ? kb : ka;
    const uint32_t* __restrict__ src_v = dir == DIR_A_TO_B ? va : vb;
    uint32_t* __restrict__ dst_v = dir == DIR_A_TO_B ? vb : va;

    for (uint32_t i = tid; i < WARPS * (RADIX + 1); i += THREADS) (&s_wcnt[0][0])[i] = 0;
    if (tid == 0) {
        s_tile = atomicAdd(&ctrl->tile_ctr[pass], 1u);
        s_abort = 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t tile_base = tile * TILE;
    const uint32_t valid = (n - tile_base) < TILE ? (n - tile_base) : TILE;
    const uint32_t shift = pass * RADIX_BITS;
    const uint32_t wofs = warp * WARP_ITEMS;

    uint32_t key[ITEMS];
    uint32_t val[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t li = wofs + j * 32 + lane;
        key[j] = li < valid ? ld_stream(src_k + tile_base + li) : 0u;
        if (PAIRS) val[j] = li < valid ? ld_stream(src_v + tile_base + li) : 0u;
    }

    uint32_t rank[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t li = wofs + j * 32 + lane;
        const uint32_t d = li < valid ? (key[j] >> shift) & (RADIX - 1) : RADIX;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader) before = atomicAdd(&s_wcnt[warp][d], (uint32_t)__popc(peers));
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[j] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();

    // Per digit: exclusive offsets of the warps and the tile's count; publish
    // the count; exclusive prefix over digits inside the tile.
    uint32_t count = 0;
    if (tid < RADIX) {
#pragma unroll
        for (uint32_t w = 0; w < WARPS; ++w) {
            const uint32_t c = s_wcnt[w][tid];
            s_wcnt[w][tid] = count;
            count += c;
        }
        const bool withhold = (debug & DBG_WITHHOLD_FIRST_TILE) && tile == 0;
        if (!withhold)
            st_relaxed(status + (size_t)tile * RADIX + tid, (tile == 0 ? SW::INC : SW::AGG) | (S)count);
    }
    uint32_t x = count;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (tid < RADIX && lane == 31) s_scan[warp] = x;
    __syncthreads();

    if (tid < RADIX) {
        uint32_t off = 0;
        for (uint32_t w = 0; w < warp; ++w) off += s_scan[w];
        const uint32_t excl_in_tile = off + x - count;
        s_excl[tid] = excl_in_tile;

        S before_tile = 0;  // items of digit tid in all earlier tiles
        if (tile > 0) {
            uint32_t t = tile - 1;
            uint32_t spins = 0;
            bool stop = false;
            while (!stop) {
                const S s = ld_relaxed(status + (size_t)t * RADIX + tid);
                const S flag = s & SW::FLAGS;
                if (flag != 0) {
                    before_tile += s & SW::VALUE;
                    if (flag == SW::INC || t == 0) break;
                    --t;
                    continue;
                }
                if (++spins > spin_limit) {
                    record_error(ctrl, sticky, ERR_TIMEOUT);
                    __threadfence();  // error visible before the INC below
                    s_abort = 1;
                    stop = true;
                } else if ((spins & 63u) == 0 && ld_relaxed(&ctrl->err) != 0) {
                    s_abort = 1;
                    stop = true;
                }
            }
            st_relaxed(status + (size_t)tile * RADIX + tid,
                       SW::INC | ((before_tile + (S)count) & SW::VALUE));
        }
        s_gofs[tid] = ctrl->gofs[pass][tid] + (uint32_t)before_tile - excl_in_tile;
    }
    if (tid == 0) {
        __threadfence();
        if (ld_relaxed(&ctrl->err) != 0) s_abort = 1;
    }
    __syncthreads();
    if (s_abort) return;

    // Stage the tile in bucket order.
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t li = wofs + j * 32 + lane;
        if (li < valid) {
            const uint32_t d = (key[j] >> shift) & (RADIX - 1);
            const uint32_t pos = s_excl[d] + s_wcnt[warp][d] + rank[j];
            s_stage[pos] = key[j];
            rank[j] = pos;
        }
    }
    __syncthreads();

    bool bad = false;
    uint32_t gpos[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint32_t s = k * THREADS + tid;
        gpos[k] = 0xffffffffu;
        if (s < valid) {
            const uint32_t kk = s_stage[s];
            const uint32_t g = s_gofs[(kk >> shift) & (RADIX - 1)] + s;
            gpos[k] = g;
            if (g < n) dst_k[g] = kk;
            else bad = true;
        }
    }
    if (PAIRS) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t li = wofs + j * 32 + lane;
            if (li < valid) s_stage[rank[j]] = val[j];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const uint32_t s = k * THREADS + tid;
            if (s < valid && gpos[k] < n) dst_v[gpos[k]] = s_stage[s];
        }
    }
    if (bad) record_error(ctrl, sticky, ERR_BOUNDS);
}

}  // namespace rs
