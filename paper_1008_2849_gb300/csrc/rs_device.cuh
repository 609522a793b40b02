// rs_device.cuh -- device-side building blocks shared by the sort kernels.
//
// Control block, status-word encoding of the decoupled look-back, relaxed
// global loads/stores, and the error bits kernels record instead of faulting.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rs {

constexpr uint32_t RADIX_BITS = 8;                 // D = 8 (Sec. 4, Alg. 2)
constexpr uint32_t RADIX = 1u << RADIX_BITS;       // 256 buckets per pass
constexpr uint32_t PASSES = 4;                     // K / D with K = 32

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
struct Ctrl {
    uint32_t err;                  // error bits of this call
    uint32_t tile_ctr[PASSES];     // dynamic tile ids, one counter per pass
    uint32_t dir[PASSES];          // pass plan
    uint32_t pad[7];               // keep hist 64-byte aligned
    uint32_t hist[PASSES][RADIX];  // digit histograms (H)
    uint32_t gofs[PASSES][RADIX];  // first output slot of every bucket (G)
};

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

__device__ __forceinline__ void record_error(Ctrl* ctrl, uint32_t* sticky, uint32_t bits) {
    atomicOr(&ctrl->err, bits);
    atomicOr(sticky, bits);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace rs
