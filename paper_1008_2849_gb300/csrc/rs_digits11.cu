// rs_digits11.cu -- the LSD sort of unsigned 32-bit keys (optionally with
// 32-bit values) with wider digits: three stable counting-sort passes of 11,
// 11 and 10 bits (Sec. 4 with D = 11: ceil(K / D) = 3 passes), against the
// four 8-bit passes of the default sort.
//
// With 2048 buckets a decoupled look-back would publish 2048 status words per
// tile (8 KB), about 256 MB per pass at 2^28 items -- more than the L2.  So
// every pass is a reduce-then-scan instead:
//   k11_up    every CTA counts the digits of its contiguous chunk of the
//             input (2048 shared counters) into counts[chunk][bucket];
//   k11_scan  per bucket, the exclusive prefix over chunks (in place) and the
//             bucket's total;
//   k11_down  every CTA sorts its chunk tile by tile:
//             A. every warp ranks the items of its slice among the warp's
//                items of the same digit, in input order (peers from one
//                ballot per digit bit; the lowest peer advances the warp's
//                16-bit counter of the digit by the group's size), keeping
//                the ranks in registers;
//             B. per bucket, the tile's count and the prefix over (bucket,
//                warp) become every warp's first tile slot of every bucket,
//                and the bucket's global offset for this tile;
//             C. every item is staged in shared memory at its tile slot,
//                so that the tile is in bucket order;
//             D. the staged tile goes out in order, every bucket run at its
//                chunk's running offset, which then advances by the tile's
//                count.
//             A chunk's first slot of bucket b is G[b] (the exclusive prefix
//             of the totals, which every CTA computes from the 2048 totals)
//             plus the chunk's prefix over chunks.
// Passes go caller -> alternate -> second alternate -> caller, so the result
// lands in the caller's arrays after three passes without a copy.
#include "rs_internal.h"
#include "rs_device.cuh"

namespace rs {

namespace {

constexpr uint32_t D11_RADIX = 2048;     // buckets of an 11-bit digit
constexpr uint32_t D11_PASSES = 3;
constexpr uint32_t D11_UP_THREADS = 1024;
constexpr uint32_t D11_UP_UNROLL = 8;    // loads in flight per thread
constexpr uint32_t D11_SCAN_GROUPS = 32; // chunk groups per bucket in k11_scan

__device__ __forceinline__ uint32_t digit11(uint32_t key, uint32_t shift) {
    return (key >> shift) & (D11_RADIX - 1);  // the last pass's top bit is 0
}

// Tile shapes of k11_down: X(index, threads, items per thread, CTAs per SM).
#define RS_D11_SHAPES(X) \
    X(0, 256, 32, 2)     \
    X(1, 512, 32, 1)     \
    X(2, 512, 16, 1)     \
    X(3, 256, 24, 2)

template <uint32_t THREADS, uint32_t ITEMS, bool PAIRS>
struct D11Shape {
    static constexpr uint32_t WARPS = THREADS / 32;
    static constexpr uint32_t TILE = THREADS * ITEMS;
    static constexpr uint32_t BPT = D11_RADIX / THREADS;  // buckets per thread in phase B
    static constexpr uint32_t WPT = BPT / 2;              // their u32 words of u16 counters
    // Shared bytes: staged keys (and values), per-warp u16 counters, per
    // bucket running offset and tile offset.
    static constexpr size_t STG = 0;
    static constexpr size_t ROWS = STG + (size_t)TILE * (PAIRS ? 8 : 4);
    static constexpr size_t RUN = ROWS + (size_t)WARPS * D11_RADIX * 2;
    static constexpr size_t OFF = RUN + D11_RADIX * 4;
    static constexpr size_t BYTES = OFF + D11_RADIX * 4;
    static_assert(BPT == 4 || BPT == 8, "phase B reads 2 or 4 counter words per row");
    static_assert(32 * ITEMS <= 65535 && TILE <= 65535, "ranks and slots fit 16 bits");
    static_assert(ITEMS % 2 == 0, "ranks are packed in pairs");
};

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(D11_UP_THREADS, 2)
k11_up(const uint32_t* __restrict__ keys, uint32_t n, uint32_t shift, uint32_t chunk,
       uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_h[D11_RADIX];
    const uint32_t tid = threadIdx.x;
    for (uint32_t b = tid; b < D11_RADIX; b += D11_UP_THREADS) s_h[b] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = lo + chunk < n ? lo + chunk : n;
    constexpr uint32_t STEP = D11_UP_THREADS * D11_UP_UNROLL;
    for (uint64_t i0 = lo; i0 < hi; i0 += STEP) {
        uint32_t k[D11_UP_UNROLL];
#pragma unroll
        for (uint32_t u = 0; u < D11_UP_UNROLL; ++u) {
            const uint64_t i = i0 + u * D11_UP_THREADS + tid;
            k[u] = i < hi ? __ldcs(keys + i) : 0u;
        }
#pragma unroll
        for (uint32_t u = 0; u < D11_UP_UNROLL; ++u)
            if (i0 + u * D11_UP_THREADS + tid < hi) atomicAdd(&s_h[digit11(k[u], shift)], 1u);
    }
    __syncthreads();
    for (uint32_t b = tid; b < D11_RADIX; b += D11_UP_THREADS)
        counts[(size_t)blockIdx.x * D11_RADIX + b] = s_h[b];
}

// counts[c][b] := sum over c' < c of counts[c'][b], and totals[b] := the
// bucket's total.  CTA = 32 buckets (threadIdx.x) x 32 contiguous chunk
// groups (threadIdx.y): group sums, their prefix over groups, then every
// group rewrites its chunks.
__global__ void __launch_bounds__(32 * D11_SCAN_GROUPS)
k11_scan(uint32_t* __restrict__ counts, uint32_t chunks, uint32_t* __restrict__ totals) {
    __shared__ uint32_t s_sum[D11_SCAN_GROUPS][33];
    const uint32_t b = blockIdx.x * 32 + threadIdx.x;
    const uint32_t y = threadIdx.y;
    const uint32_t per = (chunks + D11_SCAN_GROUPS - 1) / D11_SCAN_GROUPS;
    const uint32_t c0 = y * per < chunks ? y * per : chunks;
    const uint32_t c1 = c0 + per < chunks ? c0 + per : chunks;
    uint32_t sum = 0;
    for (uint32_t c = c0; c < c1; ++c) sum += counts[(size_t)c * D11_RADIX + b];
    s_sum[y][threadIdx.x] = sum;
    __syncthreads();
    if (y == 0) {
        uint32_t run = 0;
        for (uint32_t g = 0; g < D11_SCAN_GROUPS; ++g) {
            const uint32_t t = s_sum[g][threadIdx.x];
            s_sum[g][threadIdx.x] = run;
            run += t;
        }
        totals[b] = run;
    }
    __syncthreads();
    uint32_t run = s_sum[y][threadIdx.x];
    for (uint32_t c = c0; c < c1; ++c) {
        const uint32_t t = counts[(size_t)c * D11_RADIX + b];
        counts[(size_t)c * D11_RADIX + b] = run;
        run += t;
    }
}

// Block-wide exclusive prefix of one value per thread.
template <uint32_t WARPS>
__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t* s_warp) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t off = 0;
#pragma unroll
    for (uint32_t w = 0; w < WARPS; ++w) off += w < warp ? s_warp[w] : 0u;
    __syncthreads();  // s_warp may be rewritten by the next call
    return off + x - v;
}

// WPT u32 words (2 u16 counters each) at p, as one vector access.
template <uint32_t WPT>
__device__ __forceinline__ void ld_words(const uint16_t* p, uint32_t (&w)[WPT]) {
    if constexpr (WPT == 4) {
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        w[0] = t.x; w[1] = t.y;
    }
}
template <uint32_t WPT>
__device__ __forceinline__ void st_words(uint16_t* p, const uint32_t (&w)[WPT]) {
    if constexpr (WPT == 4)
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    else
        *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
}

template <uint32_t THREADS, uint32_t ITEMS, uint32_t MINB, bool PAIRS>
__global__ void __launch_bounds__(THREADS, MINB)
k11_down(const uint32_t* __restrict__ src_k, const uint32_t* __restrict__ src_v,
         uint32_t* __restrict__ dst_k, uint32_t* __restrict__ dst_v, uint32_t n, uint32_t shift,
         uint32_t chunk, const uint32_t* __restrict__ counts, const uint32_t* __restrict__ totals,
         uint32_t* __restrict__ sticky) {
    using S = D11Shape<THREADS, ITEMS, PAIRS>;
    constexpr uint32_t WARPS = S::WARPS, TILE = S::TILE, BPT = S::BPT, WPT = S::WPT;
    constexpr uint32_t WARP_ITEMS = 32 * ITEMS;
    extern __shared__ uint4 s_dyn[];
    char* const sm = reinterpret_cast<char*>(s_dyn);
    uint32_t* const stg_k = reinterpret_cast<uint32_t*>(sm + S::STG);
    uint2* const stg_kv = reinterpret_cast<uint2*>(sm + S::STG);
    uint16_t* const rows = reinterpret_cast<uint16_t*>(sm + S::ROWS);
    uint32_t* const run = reinterpret_cast<uint32_t*>(sm + S::RUN);
    uint32_t* const off = reinterpret_cast<uint32_t*>(sm + S::OFF);
    __shared__ uint32_t s_warp[WARPS];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t b0 = tid * BPT;  // this thread's buckets in phase B

    // Running offsets: G[b] plus this chunk's prefix over chunks.
    {
        uint32_t tot[BPT], sum = 0;
#pragma unroll
        for (uint32_t q = 0; q < BPT; ++q) {
            tot[q] = totals[b0 + q];
            sum += tot[q];
        }
        uint32_t g = block_excl<WARPS>(sum, s_warp);
#pragma unroll
        for (uint32_t q = 0; q < BPT; ++q) {
            run[b0 + q] = g + counts[(size_t)blockIdx.x * D11_RADIX + b0 + q];
            g += tot[q];
        }
    }
    constexpr uint32_t ROW_VEC4 = WARPS * D11_RADIX * 2 / 16;
    for (uint32_t i = tid; i < ROW_VEC4; i += THREADS)
        reinterpret_cast<uint4*>(rows)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    bool bad = false;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = lo + chunk < n ? lo + chunk : n;
    uint16_t* const row = rows + warp * D11_RADIX;
    for (uint64_t base = lo; base < hi; base += TILE) {
        const uint32_t valid = hi - base < TILE ? (uint32_t)(hi - base) : TILE;
        const uint32_t wofs = warp * WARP_ITEMS;
        const uint32_t left = valid > wofs ? valid - wofs : 0u;
        uint32_t k[ITEMS], v[ITEMS];
#pragma unroll
        for (uint32_t j = 0; j < ITEMS; ++j) {
            const bool live = j * 32 + lane < left;
            const uint64_t i = base + wofs + j * 32 + lane;
            k[j] = live ? __ldcs(src_k + i) : 0u;
            if (PAIRS) v[j] = live ? __ldcs(src_v + i) : 0u;
        }
        // A. Ranks within the warp, in input order.
        uint32_t rk[ITEMS / 2];
#pragma unroll
        for (uint32_t j = 0; j < ITEMS; ++j) {
            const uint32_t lv = prefix_lanes(j * 32, left);
            const uint32_t d = digit11(k[j], shift);
            const uint32_t peers = match_label<11>(d) & lv;
            const uint32_t first = __ffs(peers) - 1;
            uint32_t before = 0;
            if (lane == first) {
                before = row[d];
                row[d] = (uint16_t)(before + __popc(peers));
            }
            before = __shfl_sync(0xffffffffu, before, first & 31u);
            const uint32_t r = before + __popc(peers & lt);
            if (j & 1) rk[j / 2] |= r << 16;
            else rk[j / 2] = r;
        }
        __syncthreads();
        // B. Tile counts, tile slots of every (warp, bucket), tile offsets.
        {
            uint32_t c[BPT];
#pragma unroll
            for (uint32_t q = 0; q < BPT; ++q) c[q] = 0;
#pragma unroll
            for (uint32_t w = 0; w < WARPS; ++w) {
                uint32_t wd[WPT];
                ld_words<WPT>(rows + w * D11_RADIX + b0, wd);
#pragma unroll
                for (uint32_t q = 0; q < WPT; ++q) {
                    c[2 * q] += wd[q] & 0xffffu;
                    c[2 * q + 1] += wd[q] >> 16;
                }
            }
            uint32_t sum = 0;
#pragma unroll
            for (uint32_t q = 0; q < BPT; ++q) sum += c[q];
            uint32_t e[BPT];
            e[0] = block_excl<WARPS>(sum, s_warp);
#pragma unroll
            for (uint32_t q = 1; q < BPT; ++q) e[q] = e[q - 1] + c[q - 1];
#pragma unroll
            for (uint32_t q = 0; q < BPT; ++q) {
                const uint32_t r = run[b0 + q];
                off[b0 + q] = r - e[q];  // tile slot s of bucket b goes to off[b] + s
                run[b0 + q] = r + c[q];
            }
#pragma unroll
            for (uint32_t w = 0; w < WARPS; ++w) {
                uint32_t wd[WPT], nw[WPT];
                ld_words<WPT>(rows + w * D11_RADIX + b0, wd);
#pragma unroll
                for (uint32_t q = 0; q < WPT; ++q) {
                    nw[q] = e[2 * q] | (e[2 * q + 1] << 16);
                    e[2 * q] += wd[q] & 0xffffu;
                    e[2 * q + 1] += wd[q] >> 16;
                }
                st_words<WPT>(rows + w * D11_RADIX + b0, nw);
            }
        }
        __syncthreads();
        // C. Stage every item at its tile slot.
#pragma unroll
        for (uint32_t j = 0; j < ITEMS; ++j) {
            if (j * 32 + lane < left) {
                const uint32_t d = digit11(k[j], shift);
                const uint32_t s = row[d] + ((rk[j / 2] >> (16 * (j & 1))) & 0xffffu);
                if (s >= TILE) {
                    bad = true;
                } else if (PAIRS) {
                    stg_kv[s] = make_uint2(k[j], v[j]);
                } else {
                    stg_k[s] = k[j];
                }
            }
        }
        __syncthreads();
        // D. Counters cleared for the next tile; bucket runs out in order.
        for (uint32_t i = tid; i < ROW_VEC4; i += THREADS)
            reinterpret_cast<uint4*>(rows)[i] = make_uint4(0, 0, 0, 0);
#pragma unroll 4
        for (uint32_t s = tid; s < valid; s += THREADS) {
            uint32_t key, val = 0;
            if (PAIRS) {
                const uint2 kv = stg_kv[s];
                key = kv.x;
                val = kv.y;
            } else {
                key = stg_k[s];
            }
            const uint32_t g = off[digit11(key, shift)] + s;
            if (g < n) {
                dst_k[g] = key;
                if (PAIRS) dst_v[g] = val;
            } else {
                bad = true;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(sticky, ERR_BOUNDS);
}

struct D11Launch {
    uint32_t threads, items, tile;
    size_t smem_pairs, smem_keys;
};
#define RS_D11_INFO(I, T, J, B) \
    {T, J, T * J, D11Shape<T, J, true>::BYTES, D11Shape<T, J, false>::BYTES},
constexpr D11Launch kD11Shapes[] = {RS_D11_SHAPES(RS_D11_INFO)};
#undef RS_D11_INFO
constexpr uint32_t kNumD11Shapes = sizeof(kD11Shapes) / sizeof(kD11Shapes[0]);
// Layout sizing: no larger than the smallest tile of RS_D11_SHAPES, so that
// the counts buffer holds a chunk per tile of any shape.
constexpr uint32_t kD11MinTile = 4096;
constexpr uint32_t smallest_d11_tile() {
    uint32_t m = kD11Shapes[0].tile;
    for (uint32_t i = 1; i < kNumD11Shapes; ++i)
        if (kD11Shapes[i].tile < m) m = kD11Shapes[i].tile;
    return m;
}
static_assert(kD11MinTile <= smallest_d11_tile(), "every shape's tile is at least kD11MinTile");

template <uint32_t T, uint32_t J, uint32_t B, bool PAIRS>
rs_status launch_down(const uint32_t* sk, const uint32_t* sv, uint32_t* dk, uint32_t* dv,
                      uint32_t n, uint32_t shift, uint32_t chunk, uint32_t chunks,
                      const uint32_t* counts, const uint32_t* totals, uint32_t* sticky,
                      cudaStream_t stream) {
    constexpr size_t SMEM = D11Shape<T, J, PAIRS>::BYTES;
    auto kern = k11_down<T, J, B, PAIRS>;
    static DeviceOnce once;
    rs_status st = allow_smem_once(kern, SMEM, once);
    if (st != RS_OK) return st;
    kern<<<chunks, T, SMEM, stream>>>(sk, sv, dk, dv, n, shift, chunk, counts, totals, sticky);
    return RS_OK;
}

rs_status launch_down_shape(int shape, bool pairs, const uint32_t* sk, const uint32_t* sv,
                            uint32_t* dk, uint32_t* dv, uint32_t n, uint32_t shift,
                            uint32_t chunk, uint32_t chunks, const uint32_t* counts,
                            const uint32_t* totals, uint32_t* sticky, cudaStream_t stream) {
    switch (shape) {
#define RS_D11_CASE(I, T, J, B)                                                                \
    case I:                                                                                    \
        return pairs ? launch_down<T, J, B, true>(sk, sv, dk, dv, n, shift, chunk, chunks,     \
                                                  counts, totals, sticky, stream)              \
                     : launch_down<T, J, B, false>(sk, sv, dk, dv, n, shift, chunk, chunks,    \
                                                   counts, totals, sticky, stream);
        RS_D11_SHAPES(RS_D11_CASE)
#undef RS_D11_CASE
    default: return RS_ERR_INVALID_ARG;
    }
}

// CTAs per SM of every shape (the shared-memory plan allows that many).
constexpr uint32_t kD11CtasPerSm[] = {
#define RS_D11_MINB(I, T, J, B) B,
    RS_D11_SHAPES(RS_D11_MINB)
#undef RS_D11_MINB
};

}  // namespace

int d11_shape_count() { return (int)kNumD11Shapes; }

Layout11 layout11(size_t n, bool pairs) {
    Layout11 L{};
    const size_t tiles = (n + kD11MinTile - 1) / kD11MinTile;
    L.max_chunks = (uint32_t)(tiles < kD11MaxChunks ? tiles : kD11MaxChunks);
    size_t o = 0;
    for (int b = 0; b < 2; ++b) {
        L.alt_keys[b] = o;
        o = align_up(o + n * 4, 256);
        L.alt_vals[b] = o;
        if (pairs) o = align_up(o + n * 4, 256);
    }
    L.counts = o;
    o = align_up(o + (size_t)L.max_chunks * D11_RADIX * 4, 256);
    L.totals = o;
    o = align_up(o + D11_RADIX * 4, 256);
    L.total = o;
    return L;
}

rs_status enqueue_sort11(uint32_t* keys, uint32_t* vals, uint32_t n, cudaStream_t stream,
                         void* workspace, size_t workspace_bytes) {
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    const bool pairs = vals != nullptr;
    const Layout11 L = layout11(n, pairs);
    if (n == 0 || workspace == nullptr || workspace_bytes < L.total ||
        ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    const int shape = knobs().d11_shape;
    if (shape < 0 || shape >= (int)kNumD11Shapes) return RS_ERR_INVALID_ARG;
    char* ws = static_cast<char*>(workspace);
    uint32_t* bk[3] = {keys, reinterpret_cast<uint32_t*>(ws + L.alt_keys[0]),
                       reinterpret_cast<uint32_t*>(ws + L.alt_keys[1])};
    uint32_t* bv[3] = {vals, pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals[0]) : nullptr,
                       pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals[1]) : nullptr};
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.counts);
    uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.totals);
    // Chunks: one per resident CTA of the downsweep (at most L.max_chunks),
    // whole tiles each.
    const uint32_t tile = kD11Shapes[shape].tile;
    const uint32_t tiles = (uint32_t)(((uint64_t)n + tile - 1) / tile);
    uint32_t want = (uint32_t)di.sm_count * kD11CtasPerSm[shape];
    if (want > L.max_chunks) want = L.max_chunks;
    const uint32_t per = (tiles + want - 1) / want;
    const uint64_t chunk64 = (uint64_t)per * tile;
    const uint32_t chunks = (uint32_t)((n + chunk64 - 1) / chunk64);
    const uint32_t chunk = chunk64 > 0xffffffffull ? 0xffffffffu : (uint32_t)chunk64;
    for (uint32_t p = 0; p < D11_PASSES; ++p) {
        const uint32_t shift = 11u * p;
        const uint32_t* sk = bk[p];
        const uint32_t* sv = bv[p];
        uint32_t* dk = bk[(p + 1) % 3];
        uint32_t* dv = bv[(p + 1) % 3];
        note_launch_begin(KK_D11_UP, stream);
        k11_up<<<chunks, D11_UP_THREADS, 0, stream>>>(sk, n, shift, chunk, counts);
        note_launch_end(KK_D11_UP, stream);
        note_launch_begin(KK_D11_SCAN, stream);
        k11_scan<<<D11_RADIX / 32, dim3(32, D11_SCAN_GROUPS), 0, stream>>>(counts, chunks, totals);
        note_launch_end(KK_D11_SCAN, stream);
        note_launch_begin(KK_D11_DOWN, stream);
        st = launch_down_shape(shape, pairs, sk, sv, dk, dv, n, shift, chunk, chunks, counts,
                               totals, di.sticky, stream);
        note_launch_end(KK_D11_DOWN, stream);
        if (st != RS_OK) return st;
        if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    return RS_OK;
}

}  // namespace rs
