// rs_digits11.cu -- the LSD sort of unsigned 32-bit keys (optionally with
// 32-bit values) with wider digits: three stable counting-sort passes of 11,
// 11 and 10 bits (Sec. 4 with D = 11: ceil(K / D) = 3 passes), against the
// four 8-bit passes of the default sort.
//
// With 2048 buckets a decoupled look-back would publish 2048 status words per
// tile (8 KB), about 512 MB per pass at 2^28 items -- far more than the L2.
// So every pass is a reduce-then-scan instead:
//   k11_up    every CTA counts the digits of its contiguous chunk of the
//             input (2048 shared counters) into counts[chunk][bucket];
//   k11_scan  per bucket, the exclusive prefix over chunks (in place) and the
//             bucket's total;
//   k11_down  every CTA sorts its chunk tile by tile: the per-warp digit
//             counts of the tile, their prefix over (bucket, warp), the stable
//             rank of every item in its warp (peers from one ballot per digit
//             bit, the lowest lane advancing the digit's counter by the
//             group's size), staging in shared memory in bucket order, and
//             stores of every bucket run at its chunk's running offset, which
//             then advances by the tile's count.  A chunk's first slot of
//             bucket b is G[b] (the exclusive prefix of the totals, computed
//             by every CTA from the 2048 totals) plus its prefix over chunks.
// Passes go caller -> alternate -> second alternate -> caller, so the result
// lands in the caller's arrays after three passes without a copy.
#include "rs_internal.h"
#include "rs_device.cuh"

namespace rs {

namespace {

constexpr uint32_t D11_RADIX = 2048;           // buckets of an 11-bit digit
constexpr uint32_t D11_UP_THREADS = 1024;
constexpr uint32_t D11_THREADS = 512;          // 16 warps
constexpr uint32_t D11_ITEMS = 8;              // items per thread per tile
constexpr uint32_t D11_WARPS = D11_THREADS / 32;
constexpr uint32_t D11_TILE = D11_THREADS * D11_ITEMS;  // 4096
constexpr uint32_t D11_BPT = D11_RADIX / D11_THREADS;   // buckets per thread (4)
constexpr uint32_t D11_PASSES = 3;

// Shared plan of k11_down (32-bit words): staged (key, value) slots, per-warp
// counters, and per-bucket running offset, tile count and tile prefix.
struct D11Smem {
    static constexpr uint32_t STG = 0;                                   // [TILE] uint2
    static constexpr uint32_t ROWS = STG + 2 * D11_TILE;                 // [WARPS][RADIX]
    static constexpr uint32_t RUN = ROWS + D11_WARPS * D11_RADIX;        // [RADIX]
    static constexpr uint32_t TCNT = RUN + D11_RADIX;                    // [RADIX]
    static constexpr uint32_t TEXCL = TCNT + D11_RADIX;                  // [RADIX]
    static constexpr uint32_t WORDS = TEXCL + D11_RADIX;
    static constexpr size_t BYTES = WORDS * sizeof(uint32_t);
};
static_assert(D11Smem::BYTES + 1024 <= 232448, "one CTA's shared memory");

__device__ __forceinline__ uint32_t digit11(uint32_t key, uint32_t shift) {
    return (key >> shift) & (D11_RADIX - 1);  // the last pass's top bit is 0
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(D11_UP_THREADS)
k11_up(const uint32_t* __restrict__ keys, uint32_t n, uint32_t shift, uint32_t chunk,
       uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_h[D11_RADIX];
    const uint32_t tid = threadIdx.x;
    for (uint32_t b = tid; b < D11_RADIX; b += D11_UP_THREADS) s_h[b] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = lo + chunk < n ? lo + chunk : n;
    for (uint64_t i = lo + tid; i < hi; i += D11_UP_THREADS)
        atomicAdd(&s_h[digit11(__ldcs(keys + i), shift)], 1u);
    __syncthreads();
    for (uint32_t b = tid; b < D11_RADIX; b += D11_UP_THREADS)
        counts[(size_t)blockIdx.x * D11_RADIX + b] = s_h[b];
}

// Thread = bucket: counts[c][b] := sum over c' < c of counts[c'][b], and
// totals[b] := the bucket's total.
__global__ void __launch_bounds__(256)
k11_scan(uint32_t* __restrict__ counts, uint32_t chunks, uint32_t* __restrict__ totals) {
    const uint32_t b = blockIdx.x * 256 + threadIdx.x;
    if (b >= D11_RADIX) return;
    uint32_t run = 0;
    for (uint32_t c = 0; c < chunks; ++c) {
        const uint32_t t = counts[(size_t)c * D11_RADIX + b];
        counts[(size_t)c * D11_RADIX + b] = run;
        run += t;
    }
    totals[b] = run;
}

// Block-wide exclusive prefix of one value per thread (D11_THREADS threads).
__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t* s_warp) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x = v;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t off = 0;
    for (uint32_t w = 0; w < warp; ++w) off += s_warp[w];
    __syncthreads();  // s_warp may be rewritten by the next call
    return off + x - v;
}

// Exclusive prefix over buckets of cnt[0..RADIX) into excl (both shared;
// thread t owns the four consecutive buckets 4t..4t+3).
__device__ __forceinline__ void bucket_excl(const uint32_t* cnt, uint32_t* excl, uint32_t* s_warp) {
    const uint4 c = reinterpret_cast<const uint4*>(cnt)[threadIdx.x];
    const uint32_t e = block_excl(c.x + c.y + c.z + c.w, s_warp);
    reinterpret_cast<uint4*>(excl)[threadIdx.x] =
        make_uint4(e, e + c.x, e + c.x + c.y, e + c.x + c.y + c.z);
}

template <bool PAIRS>
__global__ void __launch_bounds__(D11_THREADS, 1)
k11_down(const uint32_t* __restrict__ src_k, const uint32_t* __restrict__ src_v,
         uint32_t* __restrict__ dst_k, uint32_t* __restrict__ dst_v, uint32_t n, uint32_t shift,
         uint32_t chunk, const uint32_t* __restrict__ counts, const uint32_t* __restrict__ totals,
         uint32_t* __restrict__ sticky) {
    using L = D11Smem;
    extern __shared__ uint4 s_dyn[];
    uint32_t* const smem = reinterpret_cast<uint32_t*>(s_dyn);
    uint2* const stg = reinterpret_cast<uint2*>(smem + L::STG);
    uint32_t* const rows = smem + L::ROWS;
    uint32_t* const run = smem + L::RUN;
    uint32_t* const tcnt = smem + L::TCNT;
    uint32_t* const texcl = smem + L::TEXCL;
    __shared__ uint32_t s_warp[D11_WARPS];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    constexpr uint32_t WARP_ITEMS = 32 * D11_ITEMS;

    // Running offsets: G[b] (exclusive prefix of the totals) plus this
    // chunk's prefix over chunks.
    for (uint32_t b = tid; b < D11_RADIX; b += D11_THREADS) tcnt[b] = totals[b];
    for (uint32_t i = tid; i < D11_WARPS * D11_RADIX / 4; i += D11_THREADS)
        reinterpret_cast<uint4*>(rows)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    bucket_excl(tcnt, run, s_warp);
    __syncthreads();
    for (uint32_t b = tid; b < D11_RADIX; b += D11_THREADS)
        run[b] += counts[(size_t)blockIdx.x * D11_RADIX + b];

    bool bad = false;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t hi = lo + chunk < n ? lo + chunk : n;
    uint32_t* const row = rows + warp * D11_RADIX;
    for (uint64_t base = lo; base < hi; base += D11_TILE) {
        const uint32_t valid = hi - base < D11_TILE ? (uint32_t)(hi - base) : D11_TILE;
        const uint32_t wofs = warp * WARP_ITEMS;
        const uint32_t left = valid > wofs ? valid - wofs : 0u;
        // This warp's slice: item j*32 + lane of the slice, in registers.
        uint32_t k[D11_ITEMS], v[D11_ITEMS];
#pragma unroll
        for (uint32_t j = 0; j < D11_ITEMS; ++j) {
            const bool live = j * 32 + lane < left;
            const uint64_t i = base + wofs + j * 32 + lane;
            k[j] = live ? __ldcs(src_k + i) : 0u;
            v[j] = PAIRS && live ? __ldcs(src_v + i) : 0u;
        }
        // Per-warp digit counts.
#pragma unroll
        for (uint32_t j = 0; j < D11_ITEMS; ++j)
            if (j * 32 + lane < left) atomicAdd(&row[digit11(k[j], shift)], 1u);
        __syncthreads();
        // Tile counts (thread t: buckets q * 512 + t) ...
#pragma unroll
        for (uint32_t q = 0; q < D11_BPT; ++q) {
            const uint32_t b = q * D11_THREADS + tid;
            uint32_t c = 0;
#pragma unroll
            for (uint32_t w = 0; w < D11_WARPS; ++w) c += rows[w * D11_RADIX + b];
            tcnt[b] = c;
        }
        __syncthreads();
        // ... their prefix over buckets ...
        bucket_excl(tcnt, texcl, s_warp);
        __syncthreads();
        // ... and every warp's first tile slot of every bucket.
#pragma unroll
        for (uint32_t q = 0; q < D11_BPT; ++q) {
            const uint32_t b = q * D11_THREADS + tid;
            uint32_t r = texcl[b];
#pragma unroll
            for (uint32_t w = 0; w < D11_WARPS; ++w) {
                const uint32_t t = rows[w * D11_RADIX + b];
                rows[w * D11_RADIX + b] = r;
                r += t;
            }
        }
        __syncthreads();
        // Stable rank in the warp, slot by slot; stage at the tile slot.
#pragma unroll
        for (uint32_t j = 0; j < D11_ITEMS; ++j) {
            const uint32_t lv = prefix_lanes(j * 32, left);
            const uint32_t d = digit11(k[j], shift);
            const uint32_t peers = match_label<11>(d) & lv;
            const uint32_t first = __ffs(peers) - 1;
            uint32_t before = 0;
            if (lane == first) before = atomicAdd(&row[d], (uint32_t)__popc(peers));
            before = __shfl_sync(0xffffffffu, before, first & 31u);
            if ((lv >> lane) & 1u) stg[before + __popc(peers & lt)] = make_uint2(k[j], v[j]);
        }
        __syncthreads();
        // Bucket runs to the chunk's running offsets.
        for (uint32_t s = tid; s < valid; s += D11_THREADS) {
            const uint2 kv = stg[s];
            const uint32_t d = digit11(kv.x, shift);
            const uint32_t g = run[d] + (s - texcl[d]);
            if (g < n) {
                dst_k[g] = kv.x;
                if (PAIRS) dst_v[g] = kv.y;
            } else {
                bad = true;
            }
        }
        __syncthreads();
        for (uint32_t b = tid; b < D11_RADIX; b += D11_THREADS) run[b] += tcnt[b];
        for (uint32_t i = tid; i < D11_WARPS * D11_RADIX / 4; i += D11_THREADS)
            reinterpret_cast<uint4*>(rows)[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
    }
    if (bad) atomicOr(sticky, ERR_BOUNDS);
}

}  // namespace

Layout11 layout11(size_t n, bool pairs) {
    Layout11 L{};
    const size_t tiles = (n + D11_TILE - 1) / D11_TILE;
    L.max_chunks = (uint32_t)(tiles < kD11MaxChunks ? tiles : kD11MaxChunks);
    size_t off = 0;
    for (int b = 0; b < 2; ++b) {
        L.alt_keys[b] = off;
        off = align_up(off + n * 4, 256);
        L.alt_vals[b] = off;
        if (pairs) off = align_up(off + n * 4, 256);
    }
    L.counts = off;
    off = align_up(off + (size_t)L.max_chunks * D11_RADIX * 4, 256);
    L.totals = off;
    off = align_up(off + D11_RADIX * 4, 256);
    L.total = off;
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
    char* ws = static_cast<char*>(workspace);
    uint32_t* bk[3] = {keys, reinterpret_cast<uint32_t*>(ws + L.alt_keys[0]),
                       reinterpret_cast<uint32_t*>(ws + L.alt_keys[1])};
    uint32_t* bv[3] = {vals, pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals[0]) : nullptr,
                       pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals[1]) : nullptr};
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.counts);
    uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.totals);
    // Chunks: at most one per SM (and at most L.max_chunks), whole tiles each.
    const uint32_t tiles = (uint32_t)((n + D11_TILE - 1) / D11_TILE);
    const uint32_t want = (uint32_t)di.sm_count < L.max_chunks ? (uint32_t)di.sm_count
                                                                : L.max_chunks;
    const uint32_t per = (tiles + want - 1) / want;
    const uint64_t chunk64 = (uint64_t)per * D11_TILE;
    const uint32_t chunks = (uint32_t)((n + chunk64 - 1) / chunk64);
    const uint32_t chunk = chunk64 > 0xffffffffull ? 0xffffffffu : (uint32_t)chunk64;
    auto down = pairs ? k11_down<true> : k11_down<false>;
    static DeviceOnce smem_set[2];
    st = allow_smem_once(down, D11Smem::BYTES, smem_set[pairs ? 1 : 0]);
    if (st != RS_OK) return st;
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
        k11_scan<<<D11_RADIX / 256, 256, 0, stream>>>(counts, chunks, totals);
        note_launch_end(KK_D11_SCAN, stream);
        note_launch_begin(KK_D11_DOWN, stream);
        down<<<chunks, D11_THREADS, D11Smem::BYTES, stream>>>(sk, sv, dk, dv, n, shift, chunk,
                                                             counts, totals, di.sticky);
        note_launch_end(KK_D11_DOWN, stream);
        if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    return RS_OK;
}

}  // namespace rs
