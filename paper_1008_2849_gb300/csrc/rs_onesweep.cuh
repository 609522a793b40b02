// rs_onesweep.cuh -- k_onesweep, one stable counting-sort pass (Sec. 3/4)
// per launch, as a persistent kernel: per-tile ranking, a decoupled
// look-back across tiles for the tile's share of every bucket, staging of the
// tile in shared memory in bucket order, and coalesced stores of every bucket
// run -- the GPU counterpart of the software write-combining buffers of
// Sec. 2.
#pragma once

#include <type_traits>

#include "rs_device.cuh"

namespace rs {

// ---------------------------------------------------------------------------
// Shared-memory plan of k_onesweep (offsets in 32-bit words; KW and VW =
// words per key and per value, 1 for 32-bit and 2 for 64-bit items):
//   in_k[2][TILE * max(KW, VW) + pad]
//                        input keys of the current and the next tile; the
//                        current tile's values are staged here once its keys
//                        are ranked
//   in_v[TILE * VW + pad] input values of the current tile (key-value sorts)
// 32-bit keys with 32-bit values (PACKED) keep one key buffer instead, and
// their stage holds (key, value) slots of 8 bytes written while ranking; the
// next tile's keys and values are copied in once the current tile is ranked.
// An input buffer holds its tile at the same offset modulo 16 bytes as in
// global memory (a skew of up to 12 bytes, hence the 16-byte pad), so that
// the tile's 16-byte-aligned middle always arrives by one bulk copy.
//   stage[TILE]          the current tile's keys in bucket order
//   wcnt[WARPS][RADIX]   per-warp digit counts of a tile, turned into per-warp
//                        tile positions while the tile is ranked
//   mask[WARPS][RADIX]   per-warp peer masks of the ranking (zero between uses)
// ---------------------------------------------------------------------------
template <int THREADS, int ITEMS, bool PAIRS, int KW = 1, int VW = 1>
struct OnesweepSmem {
    static constexpr uint32_t WARPS = THREADS / 32;
    static constexpr uint32_t TILE = THREADS * ITEMS;
    static constexpr uint32_t PAD = 4;                   // words after every input buffer
    // 32-bit keys with 32-bit values: one key buffer, and every staged slot
    // holds its key and value together (8 bytes).
    static constexpr bool PACKED = PAIRS && KW == 1 && VW == 1;
    static constexpr uint32_t BW = PAIRS && VW > KW ? VW : KW;  // words per buffer item
    static constexpr uint32_t KBUF = TILE * BW + PAD;    // words per key buffer
    static constexpr uint32_t IN_K = 0;
    static constexpr uint32_t IN_V = IN_K + (PACKED ? 1 : 2) * KBUF;
    static constexpr uint32_t STG = IN_V + (PAIRS ? TILE * VW + PAD : 0);
    static constexpr uint32_t WCNT = STG + TILE * (PACKED ? 2 : KW);
    static_assert(KBUF % 4 == 0 && (TILE * VW + PAD) % 4 == 0 && STG % KW == 0,
                  "input buffers 16-byte aligned for the bulk copies, stage aligned to keys");
    static_assert(!PACKED || STG % 2 == 0, "packed stage 8-byte aligned");
    static constexpr uint32_t MASK = WCNT + WARPS * RADIX;
    static constexpr uint32_t WORDS = MASK + WARPS * RADIX;
    static constexpr size_t BYTES = WORDS * sizeof(uint32_t);
};

// ---------------------------------------------------------------------------
// k_onesweep: one stable counting-sort pass by digit `pass` over tiles of
// TILE = THREADS * ITEMS items, run by a persistent grid.  `slot` names the
// plan entry (ctrl->dir, ctrl->tile_ctr) of the launch: the pass itself, or
// MSD_SLOT for the first pass of the MSD-first order.
//
// Tile flow inside a CTA (tile ids come from an atomic counter, in increasing
// order per CTA): while tile i is ranked, the keys of tile i+1 are already
// being copied into the other key buffer by the tensor memory accelerator
// (one bulk copy, completing on an mbarrier); tile i+1's values follow as soon
// as tile i's values have been staged.  (32-bit pairs, PACKED: both of tile
// i+1's copies start once tile i is ranked.)  A tile sits in its buffer at its
// global 16-byte phase, so the bulk copy takes its aligned middle and at most
// three items before and after it arrive by per-thread asynchronous copies on
// the same barrier.  As soon as tile i+1's keys have landed its per-warp digit
// counts are taken and its tile counts published.  Keys are 32-bit (K =
// uint32_t) or 64-bit (K = unsigned long long, eight passes); values (V) too.
//
// Item order: warp w owns tile items [w*32*ITEMS, (w+1)*32*ITEMS); its item j
// on lane l is tile item w*32*ITEMS + j*32 + l, so the (warp, j, lane) order
// is the input order -- which is what keeps the ranking stable.
//
// Per tile:
//  1. From the per-warp counts: the tile's count c[b] of every digit, its
//     exclusive prefix over digits, and every warp's first tile position for
//     every digit (warps before it come first).
//  2. Ranking (per warp, item slot j at a time): the lanes holding the same
//     digit come from one ballot per digit bit (odd slots) or from a shared
//     peer mask each lane ORs its bit into (even slots).  Alternating keeps
//     both the integer and the shared-memory pipes busy; slots go in pairs,
//     an odd slot's ballots running while the even slot before it waits for
//     its mask.  The lowest lane of a group adds the group's size to the
//     warp's position counter of the digit; an item's tile position is the
//     counter's old value plus the number of its peers on lower lanes.  The
//     key (with its value, for 32-bit pairs) is written straight to that
//     position of the staging buffer.
//  3. Look-back (threads b < 256): read the status words of the WINDOW tiles
//     before this one at once, add AGG counts from the nearest one on until an
//     INC prefix, re-reading from the first tile that has not published yet;
//     publish this tile's inclusive prefix (INC).  Meanwhile the other warps
//     count the next tile; its counts are published while this tile is
//     stored.  A CTA takes its next tile id only after its look-back (and
//     starts pulling that tile into L2), so between taking an id and
//     publishing that tile's counts it waits on no other CTA; every tile before
//     this one has therefore published its counts or will without waiting, and
//     the earliest unfinished tile always progresses.  Every wait is bounded by
//     spin_limit polls; when it runs out the kernel records ERR_TIMEOUT and
//     CTAs that see the error write nothing more.
//  4. Values are staged at the same positions (in the key buffer, free now),
//     or, for 32-bit pairs, were staged with their keys while ranking.
//  5. Slot s of the staging buffer is stored to
//       dst[G[b] + prefix_before_this_tile[b] + (s - tile_excl[b])],
//     so consecutive threads store consecutive addresses of one bucket run.
//     Threads >= 256 store most of the slots (all of them for 32-bit pairs)
//     while threads < 256 prepare the next tile (its counts, AGG and warp
//     bases).  Every global store is checked against n (ERR_BOUNDS instead
//     of a fault).
// ---------------------------------------------------------------------------
// Typed keys (TYPED; 32-bit or 64-bit): the first pass that moves data maps
// every key it reads onto its ordered unsigned word (key_to_ordered), so all
// digits, ranks and staged keys of the sort are those of the ordered words,
// and the last pass maps every key it stores back (key_from_ordered).  Values
// are untouched.
//
// Segmented sorts (SEG): tiles never straddle a segment.  tile_geo[t] =
// (first item, item count, first tile of its segment, segment) for every tile
// of the large segments; seg_gofs[s][pass][b] (pass < 4, or < 8 for 64-bit
// keys) is the absolute first output
// slot of bucket b of segment s; the number of tiles is ctrl->seg_tiles.
template <int THREADS, int ITEMS, int MIN_BLOCKS, bool PAIRS, typename S, int WINDOW, bool SEG,
          bool TYPED, typename K = uint32_t, typename V = uint32_t>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS)
k_onesweep(K* __restrict__ ka, V* __restrict__ va,
           K* __restrict__ kb, V* __restrict__ vb,
           uint32_t n, uint32_t pass, uint32_t slot, uint32_t num_tiles, Ctrl* __restrict__ ctrl,
           uint32_t* __restrict__ sticky, S* __restrict__ status, S* __restrict__ status_clear,
           uint32_t clear_words, uint32_t spin_limit, uint32_t debug,
           const uint4* __restrict__ tile_geo, const uint32_t* __restrict__ seg_gofs,
           uint32_t key_type) {
    using L = OnesweepSmem<THREADS, ITEMS, PAIRS, (int)(sizeof(K) / 4), (int)(sizeof(V) / 4)>;
    using SW = StatusWord<S>;
    static_assert(sizeof(K) == 4 || sizeof(K) == 8, "32-bit or 64-bit keys");
    static_assert(sizeof(V) == 4 || sizeof(V) == 8, "32-bit or 64-bit values");
    constexpr uint32_t NPASS = sizeof(K) == 8 ? PASSES64 : PASSES;
    static_assert(THREADS >= (int)RADIX && THREADS % 32 == 0, "one thread per digit");
    static_assert(RADIX_BITS == 8, "digits are whole bytes of the key");
    constexpr uint32_t WARPS = L::WARPS;
    constexpr uint32_t TILE = L::TILE;
    constexpr bool PACKED = L::PACKED;
    constexpr uint32_t WARP_ITEMS = 32 * ITEMS;
    constexpr int WIN = sizeof(S) == 8 ? WINDOW / 2 : WINDOW;  // same registers either way
    constexpr uint32_t LB_WARPS = RADIX / 32;                   // warps of the look-back
    constexpr bool SPARE = WARPS > LB_WARPS;                    // warps free to count meanwhile
    constexpr uint32_t ISSUER = THREADS - 1;                    // issues the bulk copies
    // Store split of the staged tile (see the scatter below): threads >= RADIX
    // do no prep of the next tile, so they start on the stores at once and
    // take a share SPLIT_NUM / 4 of the tile (at most 3 * SPLIT_NUM / 4 times
    // ITEMS each): all of it for 32-bit pairs, three quarters otherwise
    // (measured best on GB300).
    constexpr uint32_t FREE = THREADS - RADIX;
    constexpr uint32_t SPLIT_NUM = PACKED ? 4 : 3;
    constexpr uint32_t EARLY_CAP = (ITEMS * 3 * SPLIT_NUM) / 4;
    constexpr uint32_t EARLY_FIT = FREE == 0 ? 0 : (TILE * SPLIT_NUM / 4) / FREE;
    constexpr uint32_t EARLY_PER = EARLY_CAP < EARLY_FIT ? EARLY_CAP : EARLY_FIT;
    constexpr uint32_t EARLY = EARLY_PER * FREE;
    constexpr uint32_t LATE_PER = (TILE - EARLY + THREADS - 1) / THREADS;
    static_assert(L::BYTES + 4096 <= 232448, "shared memory plan exceeds one CTA's limit");

    extern __shared__ uint4 s_dyn[];
    uint32_t* const smem = reinterpret_cast<uint32_t*>(s_dyn);
    K* const s_stage = reinterpret_cast<K*>(smem + L::STG);
    // Key buffer b (as K*), not yet skewed.
    auto key_buf = [&](uint32_t b) {
        return reinterpret_cast<K*>(smem + L::IN_K + (PACKED ? 0u : b) * L::KBUF);
    };
    uint2* const s_stage2 = reinterpret_cast<uint2*>(smem + L::STG);  // PACKED: (key, value)
    uint32_t* const s_wcnt = smem + L::WCNT;
    const V* const s_in_v = reinterpret_cast<const V*>(smem + L::IN_V);
    __shared__ uint32_t s_gbase[RADIX];  // G[pass][b]
    __shared__ uint32_t s_gofs[RADIX];   // G + before_tile - tile_excl, per tile
    __shared__ uint32_t s_cnt[RADIX];    // digit counts of the next tile to rank
    __shared__ uint32_t s_excl[RADIX];   // their exclusive prefix over digits
    __shared__ uint32_t s_scan[RADIX / 32];
    __shared__ uint32_t s_ids[4];
    __shared__ uint4 s_geo[4];  // segmented: geometry of the tiles in s_ids
    __shared__ uint32_t s_flag;
    __shared__ uint32_t s_err_seen;  // the call's error word, read once per tile
    __shared__ __align__(8) uint64_t s_bar[3];  // key buffers 0 and 1, values

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // The plan, the histograms' status clearing and the pass before this
    // one are all complete from here on.
    pdl_launch_next();
    pdl_wait();
    if (key_type & (ROLE_PLAIN_PASSES | ROLE_MAP_PASSES)) {
        // One of the two instances of a typed sort's pass: keep the pass if
        // it is this instance's (an executed first or last pass needs the
        // maps; every other pass, skipped ones included, does not).
        bool first = true, last = true;
        for (uint32_t q = 0; q < NPASS; ++q) {
            if (ctrl->dir[q] == DIR_SKIP) continue;
            if (q < pass) first = false;
            if (q > pass) last = false;
        }
        const bool maps = ctrl->dir[slot] != DIR_SKIP && (first || last);
        if (maps != ((key_type & ROLE_MAP_PASSES) != 0)) return;
        key_type &= KEY_TYPE_MASK;
    }
    if (SEG) {
        if (ld_relaxed(&ctrl->err) != 0) return;  // malformed segment table: no work
        num_tiles = ctrl->seg_tiles;
    }
    const uint32_t dir = ctrl->dir[slot];
    if (dir == DIR_SKIP) {
        // No tiles in this pass: clear the whole next status array here.
        if (status_clear != nullptr)
            for (uint32_t i = blockIdx.x * THREADS + tid; i < clear_words; i += gridDim.x * THREADS)
                status_clear[i] = 0;
        return;
    }
    // Typed keys: map on reading in the first executed pass, back on storing
    // in the last one (the plan in ctrl->dir says which passes execute).
    uint32_t map_in = KEY_U32, map_out = KEY_U32;
    if (TYPED) {
        bool first = true, last = true;
        for (uint32_t q = 0; q < NPASS; ++q) {
            if (ctrl->dir[q] == DIR_SKIP) continue;
            if (q < pass) first = false;
            if (q > pass) last = false;
        }
        map_in = first ? key_type : KEY_U32;
        map_out = last ? key_type : KEY_U32;
    }
    auto read_key = [map_in](K k) -> K {
        if constexpr (TYPED) return key_to_ordered(k, map_in);
        else return k;
    };
    const K* __restrict__ src_k = dir == DIR_A_TO_B ? ka : kb;
    K* __restrict__ dst_k = dir == DIR_A_TO_B ? kb : ka;
    const V* __restrict__ src_v = dir == DIR_A_TO_B ? va : vb;
    V* __restrict__ dst_v = dir == DIR_A_TO_B ? vb : va;

    for (uint32_t i = tid; i < 2 * WARPS * RADIX / 4; i += THREADS)
        reinterpret_cast<uint4*>(s_wcnt)[i] = make_uint4(0, 0, 0, 0);  // wcnt and mask
    if (!SEG && tid < RADIX) s_gbase[tid] = ctrl->gofs[pass][tid];
    // Geometry of tile t: (first item, item count, first tile of its segment,
    // segment).
    auto load_geo = [&](uint32_t t) -> uint4 {
        if (SEG) return t < num_tiles ? tile_geo[t] : make_uint4(0, 0, 0, 0);
        const uint32_t base = t * TILE;
        return make_uint4(base, (n - base) < TILE ? (n - base) : TILE, 0u, 0u);
    };
    if (tid == 0) {
        for (int b = 0; b < 3; ++b) mbar_init(&s_bar[b], 1);
        fence_mbar_init();
        s_ids[0] = atomicAdd(&ctrl->tile_ctr[slot], 1u);
        s_geo[0] = load_geo(s_ids[0]);
        s_flag = 0;
        s_err_seen = 0;
    }
    __syncthreads();

    // Skew of a tile in its input buffer: the items from the 16-byte
    // boundary at or before the tile's first item in global memory.
    auto skew_of = [](const auto* src, uint4 g) -> uint32_t {
        using T = std::remove_cv_t<std::remove_pointer_t<decltype(src)>>;
        return (uint32_t)(((uintptr_t)(src + g.x) & 15u) / sizeof(T));
    };
    // Start copying the g.y items from src + g.x into buffer dst at the
    // tile's skew (collective): the 16-byte-aligned middle by one bulk copy,
    // the few items before and after it by per-thread copies, all completing
    // on `bar`.  Items are keys (K) or values (V).
    auto issue_copy = [&](auto* dst, const auto* src, uint4 g, uint64_t* bar) {
        using T = std::remove_cv_t<std::remove_pointer_t<decltype(src)>>;
        constexpr uint32_t PER16 = 16 / sizeof(T);  // items per 16 bytes
        const uint32_t valid = g.y;
        const T* from = src + g.x;
        T* to = dst + skew_of(src, g);  // item i lands at to[i]: same offset mod 16 B
        const uint32_t a0 = (PER16 - skew_of(src, g)) & (PER16 - 1);  // first aligned item
        const uint32_t nb = valid > a0 ? ((valid - a0) & ~(PER16 - 1)) : 0u;
        const uint32_t head = nb ? a0 : valid;  // items copied one by one: [0, head) and
        const uint32_t tail = a0 + nb;          // [tail, valid) when there is a bulk part
        if (nb < valid) {  // CTA-uniform
            bool issued = false;
            for (uint32_t i = tid; i < head; i += THREADS) {
                cp_async_elem(to + i, from + i);
                issued = true;
            }
            if (nb)
                for (uint32_t i = tail + tid; i < valid; i += THREADS) {
                    cp_async_elem(to + i, from + i);
                    issued = true;
                }
            if (issued) cp_async_mbar_arrive(bar);
            __syncthreads();  // every pending count is raised before the arrival below
        }
        if (tid == ISSUER) {
            // The buffer was last written by ordinary stores: order those
            // before the bulk copy's writes.
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, nb * (uint32_t)sizeof(T));
            if (nb) tma_load_1d(to + a0, from + a0, nb * (uint32_t)sizeof(T), bar);
        }
    };

    // One thread: start pulling tile g's aligned keys (and values) into L2,
    // so that its bulk copies, issued later, hit L2.
    auto prefetch_tile = [&](uint4 g) {
        auto pf = [&](const auto* src) {
            using T = std::remove_cv_t<std::remove_pointer_t<decltype(src)>>;
            constexpr uint32_t PER16 = 16 / sizeof(T);
            const uint32_t a0 = (PER16 - skew_of(src, g)) & (PER16 - 1);
            const uint32_t nb = g.y > a0 ? ((g.y - a0) & ~(PER16 - 1)) : 0u;
            if (nb) prefetch_l2_bulk(src + g.x + a0, nb * (uint32_t)sizeof(T));
        };
        pf(src_k);
        if (PAIRS) pf(src_v);
    };

    uint32_t phase = 0;  // bit b: parity of the next completion of s_bar[b]
    auto wait_bar = [&](uint32_t b) {
        uint32_t polls = 0;
        while (!mbar_try_wait(&s_bar[b], (phase >> b) & 1u)) {
            if (++polls > spin_limit) {
                record_error(ctrl, sticky, ERR_TIMEOUT);
                s_flag = 1;
                break;
            }
        }
        phase ^= 1u << b;
    };
    // Digit of a key: byte `pass`, picked by one byte permute (the other
    // three result bytes come from the zero operand) from the key's word
    // that holds it.
    const uint32_t dsel = 0x4440u | (pass & 3u);
    const bool high_word = pass >= 4;
    auto digit_of = [dsel, high_word](K key) {
        if constexpr (sizeof(K) == 4) {
            (void)high_word;
            return __byte_perm(key, 0u, dsel);
        } else {
            const uint32_t w = high_word ? (uint32_t)(key >> 32) : (uint32_t)key;
            return __byte_perm(w, 0u, dsel);
        }
    };
    const uint32_t wofs = warp * WARP_ITEMS;
    // Count the slots of warp w of tile g (in key buffer b) into wcnt row w.
    auto count_slots_of = [&](uint32_t b, uint4 g, uint32_t w) {
        const uint32_t valid = g.y;
        const K* keys = key_buf(b) + skew_of(src_k, g) + w * WARP_ITEMS + lane;
        uint32_t* row = s_wcnt + w * RADIX;
        if (valid == TILE) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                atomicAdd(&row[digit_of(read_key(keys[j * 32]))], 1u);
        } else {
            const uint32_t left = valid > w * WARP_ITEMS ? valid - w * WARP_ITEMS : 0u;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (j * 32 + lane < left) atomicAdd(&row[digit_of(read_key(keys[j * 32]))], 1u);
        }
    };
    // Threads < 256 only, once the per-warp counts of tile t are in wcnt:
    // publish the tile's counts (AGG, or INC for the first tile of its
    // segment), keep them and their exclusive prefix over digits for the
    // look-back, and turn wcnt into every warp's first tile position of every
    // digit.  The 256 threads synchronise among themselves (named barrier 1).
    auto prep_tile = [&](uint32_t t, uint32_t first) {
        // Up to 16 warps the counts stay in registers for the rewrite below.
        constexpr uint32_t KEPT = WARPS <= 16 ? WARPS : 1;
        uint32_t kept[KEPT];
        uint32_t c = 0;
#pragma unroll
        for (uint32_t w = 0; w < WARPS; ++w) {
            const uint32_t v = s_wcnt[w * RADIX + tid];
            if (WARPS <= 16) kept[w < KEPT ? w : 0] = v;
            c += v;
        }
        s_cnt[tid] = c;
        const bool withhold = (debug & DBG_WITHHOLD_FIRST_TILE) && t == 0;
        if (!withhold)
            st_relaxed(status + (size_t)t * RADIX + tid, (t == first ? SW::INC : SW::AGG) | (S)c);
        uint32_t x = c;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_scan[warp] = x;
        named_barrier_sync(1, RADIX);
        uint32_t off = 0;
        for (uint32_t w = 0; w < warp; ++w) off += s_scan[w];
        const uint32_t excl = off + x - c;
        s_excl[tid] = excl;
        uint32_t run = excl;
#pragma unroll
        for (uint32_t w = 0; w < WARPS; ++w) {
            const uint32_t v = WARPS <= 16 ? kept[w < KEPT ? w : 0] : s_wcnt[w * RADIX + tid];
            s_wcnt[w * RADIX + tid] = run;
            run += v;
        }
        named_barrier_sync(1, RADIX);  // s_scan may be rewritten for the next tile
    };

    // Prologue: the first tile's data and counts; the second tile's id is taken
    // once they are published.
    if (s_ids[0] >= num_tiles) return;
    issue_copy(key_buf(0), src_k, s_geo[0], &s_bar[0]);
    if (PAIRS) issue_copy(reinterpret_cast<V*>(smem + L::IN_V), src_v, s_geo[0], &s_bar[2]);
    wait_bar(0);
    count_slots_of(0, s_geo[0], warp);
    __syncthreads();
    if (tid < RADIX) prep_tile(s_ids[0], s_geo[0].z);
    if (tid == 0) {
        s_ids[1] = atomicAdd(&ctrl->tile_ctr[slot], 1u);
        s_geo[1] = load_geo(s_ids[1]);
    }
    __syncthreads();

    const uint32_t lt = lanemask_lt();

    for (uint32_t it = 0;; ++it) {
        const uint32_t tile = s_ids[it & 3];
        if (tile >= num_tiles) break;
        const uint32_t buf = it & 1;
        const uint32_t nxt = s_ids[(it + 1) & 3];
        const uint4 geo = s_geo[it & 3];
        const uint4 ngeo = s_geo[(it + 1) & 3];
        const bool have_next = nxt < num_tiles;
        if (!PACKED && have_next) issue_copy(key_buf(buf ^ 1), src_k, ngeo, &s_bar[buf ^ 1]);
        if (PACKED) wait_bar(2);  // this tile's values, read while ranking
        // Segmented: this tile's bucket bases, fetched now, used after ranking.
        uint32_t seg_base = 0;
        if (SEG && tid < RADIX) seg_base = seg_gofs[((size_t)geo.w * NPASS + pass) * RADIX + tid];
        if (tid == ISSUER) s_err_seen = ld_relaxed(&ctrl->err);
        if (status_clear != nullptr)
            for (uint32_t b = tid; b < RADIX; b += THREADS)
                status_clear[(size_t)tile * RADIX + b] = 0;

        const uint32_t valid = geo.y;
        const uint32_t first_tile = geo.z;  // look-back stops here
        K* const in_k = key_buf(buf) + skew_of(src_k, geo);
        const V* const in_v = s_in_v + (PAIRS ? skew_of(src_v, geo) : 0u);
        // Staged values: the whole key buffer is free once the keys are
        // ranked; its unskewed start is 16-byte aligned.
        V* const in_kv = reinterpret_cast<V*>(key_buf(buf));

        // ---- 2. rank, and stage the keys ------------------------------------
        uint32_t* const cnt = s_wcnt + warp * RADIX;
        uint32_t* const mask = smem + L::MASK + warp * RADIX;
        uint32_t pos[ITEMS];
        auto rank_tile = [&](auto full) {
            constexpr bool FULL = decltype(full)::value;
            const uint32_t left = FULL ? WARP_ITEMS : (valid > wofs ? valid - wofs : 0u);
            const K* keys = in_k + wofs + lane;
            auto finish = [&](int j, K k, uint32_t d, uint32_t peers, bool is_live, uint32_t val) {
                const uint32_t first = __ffs(peers) - 1;
                uint32_t before = 0;
                if (lane == first) before = atomicAdd(&cnt[d], (uint32_t)__popc(peers));
                before = __shfl_sync(0xffffffffu, before, first & 31u);
                pos[j] = before + __popc(peers & lt);
                if constexpr (PACKED) {
                    if (is_live) s_stage2[pos[j]] = make_uint2((uint32_t)k, val);
                } else {
                    if (is_live) s_stage[pos[j]] = k;
                }
            };
            const V* const vals = in_v + wofs + lane;
            K nk0 = read_key(keys[0]);
            K nk1 = ITEMS > 1 ? read_key(keys[32]) : K(0);
            uint32_t nv0 = PACKED ? (uint32_t)vals[0] : 0u;
            uint32_t nv1 = PACKED && ITEMS > 1 ? (uint32_t)vals[32] : 0u;
#pragma unroll
            for (int j = 0; j < ITEMS; j += 2) {
                // Slot j by shared-memory peer masks; slot j+1 by ballots,
                // computed while slot j's mask updates settle.  Both slots'
                // keys (and values) were read during the pair before, so the
                // loads overlap the ranking.
                const bool two = j + 1 < ITEMS;
                const bool live0 = FULL || j * 32 + lane < left;
                const K k0 = nk0, k1 = nk1;
                const uint32_t v0 = nv0, v1 = nv1;
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
                if (j + 2 < ITEMS) {  // the next pair's loads overlap this pair's tail
                    nk0 = read_key(keys[(j + 2) * 32]);
                    nk1 = j + 3 < ITEMS ? read_key(keys[(j + 3) * 32]) : K(0);
                    nv0 = PACKED ? (uint32_t)vals[(j + 2) * 32] : 0u;
                    nv1 = PACKED && j + 3 < ITEMS ? (uint32_t)vals[(j + 3) * 32] : 0u;
                }
                finish(j, k0, d0, peers0, live0, v0);
                if (two) finish(j + 1, k1, d1, peers1, live1, v1);
            }
        };
        if (valid == TILE)
            rank_tile(std::true_type{});
        else
            rank_tile(std::false_type{});
        // This warp's counter row is done: clear it for the next tile's counts.
        __syncwarp();
        for (uint32_t i = lane; i < RADIX / 4; i += 32)
            reinterpret_cast<uint4*>(cnt)[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        if (PACKED && have_next) {  // both input buffers are free now
            issue_copy(key_buf(buf ^ 1), src_k, ngeo, &s_bar[buf ^ 1]);
            issue_copy(reinterpret_cast<V*>(smem + L::IN_V), src_v, ngeo, &s_bar[2]);
        }

        // ---- 3. look-back (threads < 256) || count the next tile; values ----
        uint32_t next_id = 0;
        uint4 next_geo = make_uint4(0, 0, 0, 0);
        if (tid < RADIX) {
            const uint32_t count = s_cnt[tid];
            S before_tile = 0;
            if (tile > first_tile) {
                int32_t t = (int32_t)tile - 1;
                const int32_t lo = (int32_t)first_tile;
                uint32_t spins = 0;
                while (true) {
                    // Status words of tiles t, t-1, ..., t-WIN+1 (INC 0 before lo).
                    S lb[WIN];
                    const S* at = status + (size_t)t * RADIX + tid;
                    if (t - (WIN - 1) >= lo) {  // CTA-uniform
#pragma unroll
                        for (int i = 0; i < WIN; ++i) lb[i] = ld_relaxed(at - (size_t)i * RADIX);
                    } else {
#pragma unroll
                        for (int i = 0; i < WIN; ++i)
                            lb[i] = (t - i >= lo) ? ld_relaxed(at - (size_t)i * RADIX) : SW::INC;
                    }
                    // The walk adds the AGG words, nearest first, up to the first
                    // other word: an INC (added; the walk is done) or a word not
                    // published yet (waited for).  stop = its index, WIN if none.
                    int stop = WIN;
                    S end = 0;
#pragma unroll
                    for (int i = WIN - 1; i >= 0; --i) {
                        if ((lb[i] & SW::FLAGS) != SW::AGG) {
                            stop = i;
                            end = lb[i];
                        }
                    }
                    // Words before `stop` all carry the AGG flag: add them whole and
                    // take the flags off at once (wrap-around arithmetic).
                    S sum = 0;
#pragma unroll
                    for (int i = 0; i < WIN; ++i)
                        if (i < stop) sum += lb[i];
                    before_tile += sum - (S)stop * SW::AGG;
                    if ((end & SW::FLAGS) == SW::INC) {
                        before_tile += end & SW::VALUE;
                        break;
                    }
                    t -= stop;
                    if (stop == WIN) continue;
                    if (++spins > spin_limit) {
                        record_error(ctrl, sticky, ERR_TIMEOUT);
                        __threadfence();  // error visible before the INC below
                        s_flag = 1;
                        break;
                    }
                    if ((spins & 63u) == 0 && ld_relaxed(&ctrl->err) != 0) {
                        s_flag = 1;
                        break;
                    }
                }
                st_relaxed(status + (size_t)tile * RADIX + tid,
                           SW::INC | ((before_tile + (S)count) & SW::VALUE));
            }
            s_gofs[tid] = (SEG ? seg_base : s_gbase[tid]) + (uint32_t)before_tile - s_excl[tid];
            if (tid == 0) {
                if (s_err_seen) s_flag = 1;
                // This CTA waits on no other CTA from here until the counts of
                // the tile taken now are published: taking it cannot stall
                // anyone.
                next_id = atomicAdd(&ctrl->tile_ctr[slot], 1u);
                next_geo = load_geo(next_id);
                // 32-bit pairs copy a tile in only once the tile before it is
                // ranked: start pulling it into L2 an iteration earlier.
                if (PACKED && next_id < num_tiles) prefetch_tile(next_geo);
            }
        }
        if (have_next) {
            if (SPARE) {
                if (warp >= LB_WARPS) {
                    wait_bar(buf ^ 1);
                    for (uint32_t w = warp - LB_WARPS; w < WARPS; w += WARPS - LB_WARPS)
                        count_slots_of(buf ^ 1, ngeo, w);
                } else {
                    phase ^= 1u << (buf ^ 1);  // the count warps waited for it
                }
            } else {
                wait_bar(buf ^ 1);
                count_slots_of(buf ^ 1, ngeo, warp);
            }
        }
        // Every thread stages its own items' values (the key buffer is free).
        if (PAIRS && !PACKED) {
            wait_bar(2);
            V vv[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vv[j] = in_v[wofs + j * 32 + lane];
            if (valid == TILE) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) in_kv[pos[j]] = vv[j];
            } else {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (wofs + j * 32 + lane < valid) in_kv[pos[j]] = vv[j];
            }
        }
        __syncthreads();
        if (s_flag) {  // an error somewhere: write nothing more
            if (PACKED && have_next) wait_bar(2);  // no copy is left in flight
            break;
        }
        if (PAIRS && !PACKED && have_next)
            issue_copy(reinterpret_cast<V*>(smem + L::IN_V), src_v, ngeo, &s_bar[2]);

        // ---- 4. the next tile's counts, prefix and bases || this tile's stores
        if (have_next && tid < RADIX) prep_tile(nxt, ngeo.z);
        // Staged slots [0, EARLY) are stored by the threads that do no prep,
        // which start at once; slots [EARLY, TILE) by every thread, the prep
        // threads joining once the next tile's prep is done.
        bool bad = false;
        auto scatter_tile = [&](auto full) {
            constexpr bool FULL = decltype(full)::value;
            auto store_slot = [&](uint32_t s) {
                if (FULL || s < valid) {
                    uint2 kv = make_uint2(0u, 0u);
                    if constexpr (PACKED) kv = s_stage2[s];
                    const K kk = PACKED ? (K)kv.x : s_stage[s];
                    const uint32_t g = s_gofs[digit_of(kk)] + s;
                    if (g < n) {
                        if constexpr (TYPED) dst_k[g] = key_from_ordered(kk, map_out);
                        else dst_k[g] = kk;
                        if (PAIRS) dst_v[g] = PACKED ? (V)kv.y : in_kv[s];
                    } else {
                        bad = true;
                    }
                }
            };
            if constexpr (FREE > 0) {
                if (tid >= RADIX) {
#pragma unroll
                    for (uint32_t k = 0; k < EARLY_PER; ++k) store_slot(k * FREE + (tid - RADIX));
                }
            }
#pragma unroll
            for (uint32_t k = 0; k < LATE_PER; ++k) {
                const uint32_t s = EARLY + k * THREADS + tid;
                if ((TILE - EARLY) % THREADS == 0 || s < TILE) store_slot(s);
            }
        };
        if (valid == TILE)
            scatter_tile(std::true_type{});
        else
            scatter_tile(std::false_type{});
        if (bad) record_error(ctrl, sticky, ERR_BOUNDS);
        if (tid == 0) {
            s_ids[(it + 2) & 3] = next_id;
            s_geo[(it + 2) & 3] = next_geo;
        }
        __syncthreads();
    }
    // Every bulk copy is waited for before the loop can end, so no copy is in
    // flight into this CTA's shared memory when it exits.
}

}  // namespace rs
