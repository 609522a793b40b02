// rs_pipeline.cuh -- k_onesweep_ws: one stable counting-sort pass (Sec. 3/4)
// of 32-bit keys carrying 32-bit values, as a warp-specialised persistent
// kernel: one CTA per SM whose warps form four teams that work on different
// tiles at once and hand tiles to each other through mbarriers instead of
// CTA-wide barriers.
//
//   rank team   (RW warps)  ranks the tile (stable, per warp slice) and
//                           stages every (key, value) at its tile position
//                           in bucket order -- the write-combining buffer of
//                           Sec. 2, in shared memory;
//   count team  (CW warps)  counts the next tile's digits per rank warp,
//                           publishes the tile's counts (AGG), and turns the
//                           counts into every rank warp's first position of
//                           every digit (the tile's exclusive prefix, Sec. 3);
//   look-back   (LW warps)  decoupled look-back over the tiles before this
//                           one for the tile's share of every bucket, then
//                           publishes the inclusive prefix (INC);
//   store team  (SW warps)  stores the staged tile: slot s with digit b goes
//                           to dst[G[b] + before_tile[b] + (s - tile_excl[b])],
//                           so consecutive threads store consecutive
//                           addresses of one bucket run.
//
// Buffers: two input buffers (keys and values of a tile, filled by bulk
// copies) and two staging buffers, so that the count team counts tile k+1
// while tile k is ranked, and tile k-1 is stored while tile k is ranked.
// Count rows and tile counts are double-buffered the same way.
//
// Hand-offs, per tile k (b = k % 2, every barrier completes once per use of
// buffer b, i.e. once per two tiles; a team waits for the use two tiles back
// to be finished before it overwrites a buffer):
//   in_full[b]     bulk copies of tile k landed                -> count team
//   prep_done[b]   counts published, warp bases and tile
//                  counts in shared memory                     -> rank, look-back
//   stage_full[b]  tile k staged                               -> store team
//   gofs_ready[b]  bucket offsets of tile k known              -> store team
//                                                                (and the count
//                                                                 team, for reuse)
//   stage_empty[b] tile k stored                               -> rank team,
//                                                                 look-back team
// The rank warp that finishes a tile last takes the id of the tile two ahead
// from the atomic counter and issues its bulk copies into the input buffer
// the finished tile leaves free.  A tile id that is past the end travels the
// same way (a copy with no bytes) and makes every team leave its loop.
//
// Progress: every wait of a team on tile k is on work of a tile no later
// than k, in this CTA or (look-back) in tiles with smaller ids, and ids are
// taken in increasing order, so the earliest unfinished tile always
// progresses.  Every wait is bounded: when it runs out the kernel records
// ERR_TIMEOUT, every team leaves its loop, and the CTA waits for its own bulk
// copies in flight before it exits.  Every global store is checked against n.
#pragma once

#include <type_traits>

#include "rs_device.cuh"

namespace rs {

template <int RW, int CW, int LW, int SW, int ITEMS>
struct PipeShape {
    static constexpr uint32_t WARPS = RW + CW + LW + SW;
    static constexpr uint32_t THREADS = 32 * WARPS;
    static constexpr uint32_t WARP_ITEMS = 32 * ITEMS;
    static constexpr uint32_t TILE = RW * WARP_ITEMS;
    static constexpr uint32_t PAD = 4;                    // words after an input buffer
    static constexpr uint32_t INBUF = TILE + PAD;         // words per input buffer
    // Shared-memory plan (32-bit words).
    static constexpr uint32_t IN_K = 0;                   // [2][INBUF]
    static constexpr uint32_t IN_V = IN_K + 2 * INBUF;    // [2][INBUF]
    static constexpr uint32_t STG = IN_V + 2 * INBUF;     // [2][TILE] (key, value) slots
    static constexpr uint32_t CNT = STG + 2 * 2 * TILE;   // [2][RW][RADIX]
    static constexpr uint32_t MASK = CNT + 2 * RW * RADIX;  // [RW][RADIX]
    static constexpr uint32_t TCNT = MASK + RW * RADIX;   // [2][RADIX] tile counts
    static constexpr uint32_t TEXCL = TCNT + 2 * RADIX;   // [2][RADIX] their prefix
    static constexpr uint32_t GOFS = TEXCL + 2 * RADIX;   // [2][RADIX] store offsets
    static constexpr uint32_t WORDS = GOFS + 2 * RADIX;
    static constexpr size_t BYTES = WORDS * sizeof(uint32_t);
    static_assert(INBUF % 4 == 0 && STG % 4 == 0, "buffers 16-byte aligned");
    static_assert(CW * 32 * 2 == RADIX && LW * 32 * 2 == RADIX,
                  "count and look-back teams: two digits per thread");
    static_assert(BYTES + 2048 <= 232448, "shared memory plan exceeds one CTA's limit");
};

// 64-bit relaxed accesses of two neighbouring 32-bit status words (digits
// 2i and 2i+1): one single-copy-atomic access, so both digits of a pair are
// always published and seen together.
__device__ __forceinline__ unsigned long long ld_relaxed_pair(const uint32_t* p) {
    return ld_relaxed(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ void st_relaxed_pair(uint32_t* p, uint32_t lo, uint32_t hi) {
    st_relaxed(reinterpret_cast<unsigned long long*>(p),
               ((unsigned long long)hi << 32) | (unsigned long long)lo);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier among the first `count` threads on hardware barrier `id` that also
// returns whether `pred` held in any of them (the same answer everywhere).
__device__ __forceinline__ bool named_barrier_any(uint32_t id, uint32_t count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " barrier.cta.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r) : "r"((uint32_t)pred), "r"(id), "r"(count) : "memory");
    return r != 0;
}

template <int RW, int CW, int LW, int SW, int ITEMS, int WINDOW>
__global__ void __launch_bounds__(32 * (RW + CW + LW + SW), 1)
k_onesweep_ws(uint32_t* __restrict__ ka, uint32_t* __restrict__ va,
              uint32_t* __restrict__ kb, uint32_t* __restrict__ vb,
              uint32_t n, uint32_t pass, uint32_t slot, uint32_t num_tiles,
              Ctrl* __restrict__ ctrl, uint32_t* __restrict__ sticky,
              uint32_t* __restrict__ status, uint32_t* __restrict__ status_clear,
              uint32_t clear_words, uint32_t spin_limit, uint32_t debug) {
    using P = PipeShape<RW, CW, LW, SW, ITEMS>;
    using SWD = StatusWord<uint32_t>;
    constexpr uint32_t TILE = P::TILE;
    constexpr uint32_t WARP_ITEMS = P::WARP_ITEMS;
    constexpr uint32_t C0 = RW * 32, L0 = C0 + CW * 32, S0 = L0 + LW * 32;  // first thread of a team
    constexpr uint32_t SN = SW * 32;  // store threads
    static_assert(RADIX_BITS == 8, "digits are whole bytes of the key");

    extern __shared__ uint4 s_dyn[];
    uint32_t* const smem = reinterpret_cast<uint32_t*>(s_dyn);
    __shared__ __align__(8) uint64_t s_in_full[2], s_prep_done[2], s_stage_full[2],
        s_gofs_ready[2], s_stage_empty[2];
    __shared__ uint32_t s_tile[4];     // tile id of tile k at [k % 4]
    __shared__ uint32_t s_rdone[2];    // rank warps done with the tile in input buffer b
    __shared__ uint32_t s_nload[2];    // copies issued into input buffer b
    __shared__ uint32_t s_ncons[2];    // copies of input buffer b waited for
    __shared__ uint32_t s_scan[2][CW];
    __shared__ volatile uint32_t s_abort;

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const uint32_t dir = ctrl->dir[slot];
    if (dir == DIR_SKIP) {
        // No tiles in this pass: clear the whole next status array here.
        if (status_clear != nullptr)
            for (uint32_t i = blockIdx.x * P::THREADS + tid; i < clear_words;
                 i += gridDim.x * P::THREADS)
                status_clear[i] = 0;
        return;
    }
    const uint32_t* __restrict__ src_k = dir == DIR_A_TO_B ? ka : kb;
    uint32_t* __restrict__ dst_k = dir == DIR_A_TO_B ? kb : ka;
    const uint32_t* __restrict__ src_v = dir == DIR_A_TO_B ? va : vb;
    uint32_t* __restrict__ dst_v = dir == DIR_A_TO_B ? vb : va;

    // Digit of a key: byte `pass`, one byte permute.
    const uint32_t dsel = 0x4440u | (pass & 3u);
    auto digit_of = [dsel](uint32_t key) { return __byte_perm(key, 0u, dsel); };

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s_in_full[b], 1);
            mbar_init(&s_prep_done[b], CW);
            mbar_init(&s_stage_full[b], RW);
            mbar_init(&s_gofs_ready[b], LW);
            mbar_init(&s_stage_empty[b], SW);
            s_rdone[b] = 0;
            s_nload[b] = 0;
            s_ncons[b] = 0;
        }
        s_abort = 0;
        fence_mbar_init();
    }
    for (uint32_t i = tid; i < RW * RADIX / 4 * 3; i += P::THREADS)  // count rows and masks
        reinterpret_cast<uint4*>(smem + P::CNT)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    // Bounded wait for the completion of the phase with parity `par` of
    // `bar`; false (and the CTA aborting) if it does not come.
    auto wait_bar = [&](uint64_t* bar, uint32_t par) -> bool {
        const uint32_t limit = spin_limit * 16u > spin_limit ? spin_limit * 16u : 0xffffffffu;
        uint32_t polls = 0;
        while (!mbar_try_wait(bar, par)) {
            ++polls;
            if ((polls & 63u) == 0 && s_abort) return false;
            if (polls > limit) {
                record_error(ctrl, sticky, ERR_TIMEOUT);
                s_abort = 1;
                return false;
            }
        }
        return true;
    };

    // The same wait taken by a whole warp: every lane gets the same answer
    // (false if it failed in any lane), so the warp leaves its loop whole.
    auto wait_warp = [&](uint64_t* bar, uint32_t par) -> bool {
        return __all_sync(0xffffffffu, wait_bar(bar, par)) != 0;
    };

    // Skew of tile t in its input buffer: its first item's offset, in items,
    // from the 16-byte boundary at or before it in global memory.
    auto skew_of = [](const uint32_t* src, uint32_t t) -> uint32_t {
        return (uint32_t)(((uintptr_t)(src + (size_t)t * TILE) & 15u) / 4u);
    };
    // Whole warp: take the id of tile k and start its copies into input
    // buffer k % 2 (the 16-byte-aligned middle of the keys and of the values
    // by two bulk copies, up to three items at either end by per-lane async
    // copies), all completing on in_full[k % 2].  A tile past the end gets
    // an arrival with no bytes.
    auto issue_load = [&](uint32_t k) {
        const uint32_t b = k & 1u;
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&ctrl->tile_ctr[slot], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (lane == 0) s_tile[k & 3u] = t;
        uint32_t bytes = 0;
        uint32_t nb[2] = {0, 0}, a0[2] = {0, 0};
        if (t < num_tiles) {
            const uint32_t base = t * TILE;
            const uint32_t valid = (n - base) < TILE ? (n - base) : TILE;
            bool issued = false;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const uint32_t* src = a == 0 ? src_k : src_v;
                uint32_t* buf = smem + (a == 0 ? P::IN_K : P::IN_V) + b * P::INBUF;
                const uint32_t sk = skew_of(src, t);
                uint32_t* to = buf + sk;  // item i at to[i]: same offset mod 16 bytes
                const uint32_t* from = src + base;
                a0[a] = (4u - sk) & 3u;  // first 16-byte-aligned item
                nb[a] = valid > a0[a] ? ((valid - a0[a]) & ~3u) : 0u;
                const uint32_t head = nb[a] ? a0[a] : valid;
                const uint32_t tail = a0[a] + nb[a];
                for (uint32_t i = lane; i < head; i += 32) {
                    cp_async4(to + i, from + i);
                    issued = true;
                }
                if (nb[a])
                    for (uint32_t i = tail + lane; i < valid; i += 32) {
                        cp_async4(to + i, from + i);
                        issued = true;
                    }
                bytes += nb[a] * 4u;
            }
            if (issued) cp_async_mbar_arrive(&s_in_full[b]);
            __syncwarp();  // the per-lane copies are tracked before the arrival below
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&s_in_full[b], bytes);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const uint32_t* src = a == 0 ? src_k : src_v;
                    uint32_t* buf = smem + (a == 0 ? P::IN_K : P::IN_V) + b * P::INBUF;
                    const uint32_t sk = skew_of(src, t);
                    if (nb[a])
                        tma_load_1d(buf + sk + a0[a], src + base + a0[a], nb[a] * 4u,
                                    &s_in_full[b]);
                }
            }
        } else if (lane == 0) {
            mbar_arrive(&s_in_full[b]);
        }
        if (lane == 0) s_nload[b] += 1;
    };

    if (warp == 0) {
        issue_load(0);
        issue_load(1);
    }

    if (warp < RW) {
        // ---------------- rank team: warp r ranks slice r of every tile ----
        const uint32_t r = warp;
        const uint32_t lt = lanemask_lt();
        uint32_t* const mask = smem + P::MASK + r * RADIX;
        for (uint32_t k = 0;; ++k) {
            const uint32_t b = k & 1u, par = (k >> 1) & 1u;
            if (!wait_warp(&s_prep_done[b], par)) break;
            const uint32_t t = s_tile[k & 3u];
            if (k >= 2 && !wait_warp(&s_stage_empty[b], par ^ 1u)) break;
            if (t >= num_tiles) {  // past the end: tell the store team
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_stage_full[b]);
                break;
            }
            const uint32_t base = t * TILE;
            const uint32_t valid = (n - base) < TILE ? (n - base) : TILE;
            const uint32_t* const keys =
                smem + P::IN_K + b * P::INBUF + skew_of(src_k, t) + r * WARP_ITEMS + lane;
            const uint32_t* const vals =
                smem + P::IN_V + b * P::INBUF + skew_of(src_v, t) + r * WARP_ITEMS + lane;
            uint32_t* const cnt = smem + P::CNT + (b * RW + r) * RADIX;
            uint2* const stg = reinterpret_cast<uint2*>(smem + P::STG) + b * TILE;
            auto rank_slice = [&](auto full) {
                constexpr bool FULL = decltype(full)::value;
                const uint32_t left =
                    FULL ? WARP_ITEMS : (valid > r * WARP_ITEMS ? valid - r * WARP_ITEMS : 0u);
                auto finish = [&](uint32_t k0, uint32_t d, uint32_t peers, bool live, uint32_t v) {
                    const uint32_t first = __ffs(peers) - 1;
                    uint32_t before = 0;
                    if (lane == first) before = atomicAdd(&cnt[d], (uint32_t)__popc(peers));
                    before = __shfl_sync(0xffffffffu, before, first & 31u);
                    if (live) stg[before + __popc(peers & lt)] = make_uint2(k0, v);
                };
                uint32_t nk0 = keys[0], nk1 = ITEMS > 1 ? keys[32] : 0u;
                uint32_t nv0 = vals[0], nv1 = ITEMS > 1 ? vals[32] : 0u;
#pragma unroll
                for (int j = 0; j < ITEMS; j += 2) {
                    // Slot j by shared peer masks, slot j+1 by ballots computed
                    // while slot j's mask updates settle; the next pair's keys
                    // and values load during this pair's tail.
                    const bool two = j + 1 < ITEMS;
                    const bool live0 = FULL || j * 32 + lane < left;
                    const uint32_t k0 = nk0, k1 = nk1, v0 = nv0, v1 = nv1;
                    const uint32_t d0 = digit_of(k0);
                    __syncwarp();
                    if (live0) atomicOr(&mask[d0], 1u << lane);
                    uint32_t d1 = 0, peers1 = 0;
                    bool live1 = false;
                    if (two) {
                        live1 = FULL || (j + 1) * 32 + lane < left;
                        const uint32_t lv1 = FULL ? 0xffffffffu : prefix_lanes((j + 1) * 32, left);
                        d1 = digit_of(k1);
                        peers1 = match_label<RADIX_BITS>(d1) & lv1;
                    }
                    __syncwarp();
                    const uint32_t peers0 = live0 ? mask[d0] : 0u;
                    __syncwarp();
                    if (live0 && (peers0 & lt) == 0) mask[d0] = 0;
                    if (j + 2 < ITEMS) {
                        nk0 = keys[(j + 2) * 32];
                        nk1 = j + 3 < ITEMS ? keys[(j + 3) * 32] : 0u;
                        nv0 = vals[(j + 2) * 32];
                        nv1 = j + 3 < ITEMS ? vals[(j + 3) * 32] : 0u;
                    }
                    finish(k0, d0, peers0, live0, v0);
                    if (two) finish(k1, d1, peers1, live1, v1);
                }
            };
            if (valid == TILE)
                rank_slice(std::true_type{});
            else
                rank_slice(std::false_type{});
            // This warp's count row of buffer b is done: clear it for tile k+2.
            __syncwarp();
            for (uint32_t i = lane; i < RADIX / 4; i += 32)
                reinterpret_cast<uint4*>(cnt)[i] = make_uint4(0, 0, 0, 0);
            __syncwarp();
            uint32_t last = 0;
            if (lane == 0) {
                mbar_arrive(&s_stage_full[b]);
                __threadfence_block();  // this warp's reads of input buffer b are done
                last = atomicAdd(&s_rdone[b], 1u) == RW - 1 ? 1u : 0u;
                __threadfence_block();
                if (last) s_rdone[b] = 0;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) issue_load(k + 2);  // input buffer b is free: tile k+2
        }
    } else if (warp < RW + CW) {
        // ---------------- count team: counts, AGG, warp bases ---------------
        const uint32_t c = tid - C0, cw = warp - RW;
        const uint32_t d0 = 2 * c;  // this thread's digits: d0, d0 + 1
        for (uint32_t k = 0;; ++k) {
            const uint32_t b = k & 1u, par = (k >> 1) & 1u;
            // The team leaves its loop whole (it meets at named barriers below).
            bool ok = wait_bar(&s_in_full[b], par);
            if (c == 0 && ok) s_ncons[b] += 1;
            // The look-back team is done with this buffer's tile counts (tile k-2).
            if (ok && k >= 2) ok = wait_bar(&s_gofs_ready[b], par ^ 1u);
            if (named_barrier_any(1, CW * 32, !ok)) break;
            const uint32_t t = s_tile[k & 3u];
            if (t >= num_tiles) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_prep_done[b]);
                break;
            }
            const uint32_t base = t * TILE;
            const uint32_t valid = (n - base) < TILE ? (n - base) : TILE;
            const uint32_t* const in_k = smem + P::IN_K + b * P::INBUF + skew_of(src_k, t);
            uint32_t* const rows = smem + P::CNT + b * RW * RADIX;
            for (uint32_t r = cw; r < RW; r += CW) {
                const uint32_t* keys = in_k + r * WARP_ITEMS + lane;
                uint32_t* row = rows + r * RADIX;
                if (valid == TILE) {
#pragma unroll
                    for (int j = 0; j < ITEMS; ++j) atomicAdd(&row[digit_of(keys[j * 32])], 1u);
                } else {
                    const uint32_t left = valid > r * WARP_ITEMS ? valid - r * WARP_ITEMS : 0u;
#pragma unroll
                    for (int j = 0; j < ITEMS; ++j)
                        if (j * 32 + lane < left) atomicAdd(&row[digit_of(keys[j * 32])], 1u);
                }
            }
            named_barrier_sync(1, CW * 32);  // every row of the tile is counted
            uint2 kept[RW];
            uint32_t c0 = 0, c1 = 0;
#pragma unroll
            for (uint32_t r = 0; r < RW; ++r) {
                kept[r] = *reinterpret_cast<const uint2*>(rows + r * RADIX + d0);
                c0 += kept[r].x;
                c1 += kept[r].y;
            }
            const bool withhold = (debug & DBG_WITHHOLD_FIRST_TILE) && t == 0;
            if (!withhold)
                st_relaxed_pair(status + (size_t)t * RADIX + d0,
                                (t == 0 ? SWD::INC : SWD::AGG) | c0,
                                (t == 0 ? SWD::INC : SWD::AGG) | c1);
            const uint32_t pair = c0 + c1;
            uint32_t x = pair;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_scan[b][cw] = x;
            named_barrier_sync(1, CW * 32);
            uint32_t off = 0;
            for (uint32_t w = 0; w < cw; ++w) off += s_scan[b][w];
            const uint32_t e0 = off + x - pair, e1 = e0 + c0;
            smem[P::TCNT + b * RADIX + d0] = c0;
            smem[P::TCNT + b * RADIX + d0 + 1] = c1;
            smem[P::TEXCL + b * RADIX + d0] = e0;
            smem[P::TEXCL + b * RADIX + d0 + 1] = e1;
            uint32_t run0 = e0, run1 = e1;
#pragma unroll
            for (uint32_t r = 0; r < RW; ++r) {
                *reinterpret_cast<uint2*>(rows + r * RADIX + d0) = make_uint2(run0, run1);
                run0 += kept[r].x;
                run1 += kept[r].y;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_prep_done[b]);
        }
    } else if (warp < RW + CW + LW) {
        // ---------------- look-back team -----------------------------------
        const uint32_t l = tid - L0;
        const uint32_t d0 = 2 * l;
        const uint32_t g0 = ctrl->gofs[pass][d0], g1 = ctrl->gofs[pass][d0 + 1];
        for (uint32_t k = 0;; ++k) {
            const uint32_t b = k & 1u, par = (k >> 1) & 1u;
            if (!wait_warp(&s_prep_done[b], par)) break;
            const uint32_t t = s_tile[k & 3u];
            if (t >= num_tiles) break;
            if (__any_sync(0xffffffffu, ld_relaxed(&ctrl->err) != 0)) {
                s_abort = 1;  // an error elsewhere: write nothing more
                break;
            }
            if (status_clear != nullptr) st_relaxed_pair(status_clear + (size_t)t * RADIX + d0, 0, 0);
            const uint32_t c0 = smem[P::TCNT + b * RADIX + d0];
            const uint32_t c1 = smem[P::TCNT + b * RADIX + d0 + 1];
            uint32_t bef0 = 0, bef1 = 0;
            bool ok = true;
            if (t > 0) {
                // Status pairs of tiles q, q-1, ..., q-WINDOW+1 (INC 0 before
                // tile 0); add the AGG pairs from the nearest one on up to
                // the first other pair: an INC (added; done) or one not
                // published yet (read again).
                int32_t q = (int32_t)t - 1;
                uint32_t spins = 0;
                while (true) {
                    unsigned long long lb[WINDOW];
                    const uint32_t* at = status + (size_t)q * RADIX + d0;
#pragma unroll
                    for (int i = 0; i < WINDOW; ++i)
                        lb[i] = (q - i >= 0) ? ld_relaxed_pair(at - (size_t)i * RADIX)
                                             : (unsigned long long)SWD::INC;
                    int stop = WINDOW;
                    unsigned long long end = 0;
#pragma unroll
                    for (int i = WINDOW - 1; i >= 0; --i)
                        if (((uint32_t)lb[i] & SWD::FLAGS) != SWD::AGG) {
                            stop = i;
                            end = lb[i];
                        }
                    uint32_t s0 = 0, s1 = 0;
#pragma unroll
                    for (int i = 0; i < WINDOW; ++i)
                        if (i < stop) {
                            s0 += (uint32_t)lb[i];
                            s1 += (uint32_t)(lb[i] >> 32);
                        }
                    // Every added word carries the AGG flag: take the flags off
                    // at once (wrap-around arithmetic).
                    bef0 += s0 - (uint32_t)stop * SWD::AGG;
                    bef1 += s1 - (uint32_t)stop * SWD::AGG;
                    if (((uint32_t)end & SWD::FLAGS) == SWD::INC) {
                        bef0 += (uint32_t)end & SWD::VALUE;
                        bef1 += (uint32_t)(end >> 32) & SWD::VALUE;
                        break;
                    }
                    q -= stop;
                    if (stop == WINDOW) continue;
                    if (++spins > spin_limit) {
                        record_error(ctrl, sticky, ERR_TIMEOUT);
                        __threadfence();  // the error is visible before the INC below
                        s_abort = 1;
                        ok = false;
                        break;
                    }
                    if ((spins & 63u) == 0 && (s_abort || ld_relaxed(&ctrl->err) != 0)) {
                        s_abort = 1;
                        ok = false;
                        break;
                    }
                }
                st_relaxed_pair(status + (size_t)t * RADIX + d0,
                                SWD::INC | ((bef0 + c0) & SWD::VALUE),
                                SWD::INC | ((bef1 + c1) & SWD::VALUE));
            }
            if (!__all_sync(0xffffffffu, ok)) break;
            // The store team is done with this buffer's offsets (tile k-2).
            if (k >= 2 && !wait_warp(&s_stage_empty[b], par ^ 1u)) break;
            smem[P::GOFS + b * RADIX + d0] = g0 + bef0 - smem[P::TEXCL + b * RADIX + d0];
            smem[P::GOFS + b * RADIX + d0 + 1] = g1 + bef1 - smem[P::TEXCL + b * RADIX + d0 + 1];
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_gofs_ready[b]);
        }
    } else {
        // ---------------- store team ---------------------------------------
        const uint32_t st = tid - S0;
        bool bad = false;
        for (uint32_t k = 0;; ++k) {
            const uint32_t b = k & 1u, par = (k >> 1) & 1u;
            if (!wait_warp(&s_stage_full[b], par)) break;
            const uint32_t t = s_tile[k & 3u];
            if (t >= num_tiles) break;
            if (!wait_warp(&s_gofs_ready[b], par)) break;
            const uint32_t base = t * TILE;
            const uint32_t valid = (n - base) < TILE ? (n - base) : TILE;
            const uint2* const stg = reinterpret_cast<const uint2*>(smem + P::STG) + b * TILE;
            const uint32_t* const gofs = smem + P::GOFS + b * RADIX;
            auto store_slot = [&](uint32_t s) {
                const uint2 kv = stg[s];
                const uint32_t g = gofs[digit_of(kv.x)] + s;
                if (g < n) {
                    dst_k[g] = kv.x;
                    dst_v[g] = kv.y;
                } else {
                    bad = true;
                }
            };
            if (valid == TILE) {
#pragma unroll 14
                for (uint32_t s = st; s < TILE; s += SN) store_slot(s);
            } else {
                for (uint32_t s = st; s < valid; s += SN) store_slot(s);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_stage_empty[b]);
        }
        if (bad) record_error(ctrl, sticky, ERR_BOUNDS);
    }

    // Every team has left its loop.  Wait for the bulk copies still in flight
    // into this CTA's shared memory (issued, never waited for after an
    // abort) before the CTA exits.
    __syncthreads();
    if (tid == 0) {
        for (uint32_t b = 0; b < 2; ++b) {
            if (s_nload[b] > s_ncons[b]) {
                const uint32_t par = (s_nload[b] - 1u) & 1u;
                uint32_t polls = 0;
                while (!mbar_try_wait(&s_in_full[b], par) && ++polls < (1u << 26)) {
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace rs
