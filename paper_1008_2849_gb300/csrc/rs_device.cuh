// rs_device.cuh -- device-side building blocks shared by the sort kernels.
//
// Control block, status-word encoding of the decoupled look-back, relaxed
// global loads/stores, and the error bits kernels record instead of faulting.
#pragma once

#include <cstddef>

#include <cstdint>
#include <cuda_runtime.h>

namespace rs {

constexpr uint32_t RADIX_BITS = 8;                 // D = 8 (Sec. 4, Alg. 2)
constexpr uint32_t RADIX = 1u << RADIX_BITS;       // 256 buckets per pass
constexpr uint32_t PASSES = 4;                     // K / D with K = 32
constexpr uint32_t PASSES64 = 8;                   // K / D with K = 64 (64-bit keys)

// Error bits recorded on the device: in ctrl->err for the running call and
// in the per-device sticky word that rs_stream_status reads and clears (its
// address reaches the kernels as an argument).  Kernels set a bit and stop
// doing work; they never trap.
constexpr uint32_t ERR_TIMEOUT = 1u;
constexpr uint32_t ERR_BOUNDS = 2u;
constexpr uint32_t ERR_SEGMENTS = 4u;

// Debug switches passed to the scatter kernels.
constexpr uint32_t DBG_WITHHOLD_FIRST_TILE = 1u;

// Pass plan written by the plan kernel: per pass, skip or direction.
constexpr uint32_t DIR_SKIP = 0;   // every key has the same digit: identity
constexpr uint32_t DIR_A_TO_B = 1; // caller's arrays -> alternate buffers
constexpr uint32_t DIR_B_TO_A = 2; // alternate buffers -> caller's arrays

// Per-call control block, zeroed by one cudaMemsetAsync at the start of a
// call.  Lives at the start of the workspace.
// Plan slots: the LSD passes 0..7 (0..3 for 32-bit keys), and MSD_SLOT for
// the most-significant-digit pass of the MSD-first order (Alg. 2), which runs
// before the passes 0..3 are reached and, when the plan chooses it, makes them
// all DIR_SKIP.
constexpr uint32_t MSD_SLOT = PASSES64;
constexpr uint32_t PLAN_SLOTS = PASSES64 + 1;

struct Ctrl {
    uint32_t err;                  // error bits of this call
    uint32_t tile_ctr[PLAN_SLOTS]; // dynamic tile ids, one counter per plan slot
    uint32_t dir[PLAN_SLOTS];      // pass plan
    uint32_t seg_tiles;            // segmented sorts: tiles of the large segments
    uint32_t small_count;          // segmented sorts (and MSD buckets): one-CTA segments
    uint32_t large_count;          // segmented sorts: number of large segments
    uint32_t tiny_count;           // segmented sorts (and MSD buckets): one-warp segments
    uint32_t pad[9];               // keep hist 64-byte aligned
    uint32_t hist[PASSES64][RADIX];  // digit histograms (H); 0..3 for 32-bit keys
    uint32_t gofs[PASSES64][RADIX];  // first output slot of every bucket (G)
};
static_assert(offsetof(Ctrl, hist) % 64 == 0, "histograms 64-byte aligned");

// Key types.  A typed key is mapped onto an unsigned word with the same
// order before its digits are read, and mapped back when it is stored:
//   KEY_I32  two's-complement integers by value: flip the sign bit;
//   KEY_F32  IEEE-754 binary32 by totalOrder (IEEE 754-2008 Sec. 5.10): a
//            positive-signed word gets its sign bit set, a negative-signed
//            word is complemented (larger magnitude -> smaller word).
// Both maps are bijections on 32-bit words, so sorting the mapped words
// stably and mapping back is the stable sort in the typed order.  KEY_I64 and
// KEY_F64 are the same maps on 64-bit words (bit 63 is the sign bit); KEY_U32
// (and KEY_U64) is the identity on either width.
constexpr uint32_t KEY_U32 = 0;
constexpr uint32_t KEY_I32 = 1;
constexpr uint32_t KEY_F32 = 2;
constexpr uint32_t KEY_U64 = 3;
constexpr uint32_t KEY_I64 = 4;
constexpr uint32_t KEY_F64 = 5;
// Typed sorts launch two instances of a scatter pass: one without the key
// maps, for the passes that move ordered words only, and one with them, for
// the first and the last executed pass.  Which passes those are is known on
// the device (the pass plan), so each instance returns at once unless the
// pass is its own; these bits, added to the key type argument, say which
// instance a launch is.
constexpr uint32_t ROLE_PLAIN_PASSES = 1u << 8;
constexpr uint32_t ROLE_MAP_PASSES = 1u << 9;
constexpr uint32_t KEY_TYPE_MASK = 0xffu;

__device__ __forceinline__ uint32_t key_to_ordered(uint32_t k, uint32_t type) {
    const uint32_t neg = type == KEY_F32 ? (uint32_t)((int32_t)k >> 31) : 0u;
    return k ^ (neg | (type != KEY_U32 ? 0x80000000u : 0u));
}
__device__ __forceinline__ uint32_t key_from_ordered(uint32_t k, uint32_t type) {
    const uint32_t neg = type == KEY_F32 ? ~(uint32_t)((int32_t)k >> 31) : 0u;
    return k ^ (neg | (type != KEY_U32 ? 0x80000000u : 0u));
}
__device__ __forceinline__ unsigned long long key_to_ordered(unsigned long long k, uint32_t type) {
    const unsigned long long neg =
        type == KEY_F64 ? (unsigned long long)((long long)k >> 63) : 0ull;
    return k ^ (neg | (type == KEY_I64 || type == KEY_F64 ? 0x8000000000000000ull : 0ull));
}
__device__ __forceinline__ unsigned long long key_from_ordered(unsigned long long k,
                                                               uint32_t type) {
    const unsigned long long neg =
        type == KEY_F64 ? ~(unsigned long long)((long long)k >> 63) : 0ull;
    return k ^ (neg | (type == KEY_I64 || type == KEY_F64 ? 0x8000000000000000ull : 0ull));
}

// Status words of the decoupled look-back: a 2-bit flag above a count.
//   flag 0 = nothing published, AGG = this tile's own count,
//   INC = inclusive prefix over this tile and all tiles before it.
template <typename S> struct StatusWord;
template <> struct StatusWord<uint32_t> {
    static constexpr uint32_t AGG = 1u << 30;
    static constexpr uint32_t INC = 2u << 30;
    static constexpr uint32_t FLAGS = 3u << 30;
    static constexpr uint32_t VALUE = (1u << 30) - 1u;
};
template <> struct StatusWord<unsigned long long> {
    static constexpr unsigned long long AGG = 1ull << 62;
    static constexpr unsigned long long INC = 2ull << 62;
    static constexpr unsigned long long FLAGS = 3ull << 62;
    static constexpr unsigned long long VALUE = (1ull << 62) - 1ull;
};

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Streaming load: the data is read exactly once per pass, so ask for it to be
// evicted first and not to displace the lines where scattered writes merge.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcs(p); }

// Asynchronous 4-byte global -> shared copy (no register staging); completes
// at cp_async_wait_all().
__device__ __forceinline__ void cp_async4(uint32_t* smem_dst, const uint32_t* gmem_src) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned long long* smem_dst,
                                          const unsigned long long* gmem_src) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src) : "memory");
}
// The same copy for either key width.
__device__ __forceinline__ void cp_async_elem(uint32_t* d, const uint32_t* s) { cp_async4(d, s); }
__device__ __forceinline__ void cp_async_elem(unsigned long long* d, const unsigned long long* s) {
    cp_async8(d, s);
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---- mbarrier and TMA bulk copies (sm_90+ async proxy) --------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Order this thread's earlier ordinary shared-memory accesses before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes) : "memory");
}
// Arrive on `bar` once all of this thread's earlier cp.async copies are done.
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// One bulk copy global -> shared, completing `bytes` of the barrier's
// transaction count.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(smem_dst)), "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Start pulling `bytes` (a multiple of 16) from gmem_src (16-byte aligned)
// into L2, without waiting; a later copy of the same bytes then hits L2.
__device__ __forceinline__ void prefetch_l2_bulk(const void* gmem_src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gmem_src), "r"(bytes)
                 : "memory");
}

// Barrier among the first `count` threads of the CTA (count a multiple of
// 32), on hardware barrier `id` (0 is the one __syncthreads uses).
__device__ __forceinline__ void named_barrier_sync(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialization attribute (launch_after_previous) may become resident
// while the kernel before it on the stream is still running; pdl_wait()
// returns once that kernel has completed and its writes are visible, and
// must come before anything that reads them.  (Launched without the
// attribute, the kernel starts after its predecessor and pdl_wait() returns
// at once.)  pdl_launch_next() lets the next such kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void record_error(Ctrl* ctrl, uint32_t* sticky, uint32_t bits) {
    atomicOr(&ctrl->err, bits);
    atomicOr(sticky, bits);
}

// Lanes of the warp whose BITS-bit label equals this lane's label, built from
// one ballot per label bit: a lane keeps the lanes that agree with it on
// every bit.  (The native match instruction is far slower on this part.)
template <int BITS>
__device__ __forceinline__ uint32_t match_label(uint32_t label) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const uint32_t bit = (label >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= m ^ (bit - 1u);  // bit = 1: m; bit = 0: ~m
    }
    return peers;
}

// Lanes l of the warp for which base + l < limit (a prefix of the warp).
__device__ __forceinline__ uint32_t prefix_lanes(uint32_t base, uint32_t limit) {
    if (limit <= base) return 0u;
    const uint32_t k = limit - base;
    return k >= 32u ? 0xffffffffu : ((1u << k) - 1u);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace rs
