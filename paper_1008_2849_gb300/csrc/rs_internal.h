// rs_internal.h -- host-side interface between the C ABI (rs_api.cu) and the
// kernel launchers (rs_sort.cu, rs_onesweep_*.cu).  Not installed, not part
// of the ABI.
#pragma once

#include <atomic>
#include <utility>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rs.h"

namespace rs {

struct Ctrl;

// Kernel kinds, for launch counting and per-kind event timing.
enum KernelKind : int {
    KK_HIST = 0,
    KK_PLAN = 1,
    KK_ONESWEEP = 2,
    KK_SMALL = 3,
    KK_SEG_PLAN = 4,
    KK_SEG_HIST = 5,
    KK_SEG_SCAN = 6,
    KK_SEG_ONESWEEP = 7,
    KK_WARP = 8,
    KK_D11_UP = 9,
    KK_D11_SCAN = 10,
    KK_D11_DOWN = 11,
    KK_COUNT
};
const char* kernel_kind_name(int kind);

// Called around every kernel launch by the launchers.
void note_launch_begin(int kind, cudaStream_t stream);
void note_launch_end(int kind, cudaStream_t stream);

// Tile shapes of the scatter kernel that this build instantiates:
// X(index, threads, items per thread, CTAs per SM the register budget is
// sized for, look-back window in status words).  The launchers and the host
// tables are both generated from this one list.
#define RS_TILE_SHAPES(X)   \
    X(0, 512, 16, 1, 32)    \
    X(1, 512, 8, 2, 16)     \
    X(2, 256, 16, 2, 32)    \
    X(3, 384, 13, 2, 6)     \
    X(4, 384, 12, 2, 8)     \
    X(5, 1024, 8, 1, 32)    \
    X(6, 384, 18, 2, 8)

struct TileConfig {
    int threads;
    int items;
    int min_blocks;  // CTAs per SM the register budget is sized for
    int window;      // look-back window (status words read per round trip)
};
#define RS_COUNT_SHAPE(I, T, J, B, W) +1
constexpr int NUM_TILE_CONFIGS = 0 RS_TILE_SHAPES(RS_COUNT_SHAPE);
#undef RS_COUNT_SHAPE
extern const TileConfig kTileConfigs[NUM_TILE_CONFIGS];
int smallest_tile();
// Sorts of typed keys run their scatter passes with this shape (the default
// of large arrays); only it is compiled with the key maps.
constexpr int kTypedShape = 3;

// Per size class tuning (chosen by the autotuner): tile shapes (indices into
// kTileConfigs), the largest array / segment sorted by the one-warp sort and
// by the one-CTA sort, and the digit width of those two sorts.
struct ClassKnobs {
    int tile_pairs;
    int tile_keys;
    int tile_seg;
    int small_max;
    int warp_max;
    int small_bits;
    int msd;        // 1: whole arrays up to kMsdMaxItems may take the MSD-first order
    int digits;     // 8: four 8-bit passes; 11: three 11/11/10-bit passes (rs_digits11.cu)
                    // for unsigned keys, when the caller's workspace holds their buffers
};
// Largest whole array the MSD-first order is tried for: 256 buckets of at
// most the one-CTA sort's capacity.
constexpr uint32_t kMsdMaxItems = 256u * 8192u;
// Size classes by item count (whole array; for a segmented sort the average
// segment): <= 2^13, <= 2^16, <= 2^20, <= 2^24, <= 2^28, larger.
constexpr int NUM_SIZE_CLASSES = 6;
int size_class(size_t items);

// Host-side knobs shared by every launch.
struct Knobs {
    ClassKnobs cls[NUM_SIZE_CLASSES];
    uint32_t spin_limit;     // polls per look-back wait before ERR_TIMEOUT
    uint32_t debug;          // DBG_* bits
    int hist_ctas_per_sm;
    int hist_mode;           // HIST_ATOMIC / HIST_LEADER / HIST_MATCH
    // Typed keys: sorts of at least this many items launch two instances of
    // every scatter pass (the passes that need no key map run without it);
    // smaller ones launch only the mapping instance, which runs every pass.
    uint32_t typed_split_min;
    int d11_shape;           // tile shape of the 11-bit-digit sort's scatter kernel
    int pdl;                 // 1: the plan and scatter kernels launch as programmatic dependents
};
Knobs& knobs();
// Whether a typed sort of n items launches two instances of every scatter
// pass (see Knobs::typed_split_min).
inline bool typed_split(size_t n) { return n >= knobs().typed_split_min; }

// Host-side checks shared by the sort entry points: size, null pointers,
// 4-byte alignment, keys and values not overlapping.
rs_status check_sort_args(const uint32_t* keys, const uint32_t* vals, size_t n);

// Per-device facts cached on first use.
struct DeviceInfo {
    int sm_count;
    uint32_t* sticky;        // device address of the sticky error word
};
rs_status device_info(DeviceInfo* out);

// Workspace layout of an unsegmented sort of n items.
struct Layout {
    size_t ctrl, status0, status1, alt_keys, alt_vals, msd_off, msd_tiny, msd_small, total;
    uint32_t tiles;          // tiles of the smallest tile shape (status sizing)
    bool wide_status;        // 64-bit status words (n >= 2^30)
};
Layout layout_for(size_t n, bool pairs);
// Workspace of the whole-array sorts of n items: the 8-bit layout, or the
// 11-bit one's when n's size class takes that order and it is larger.
size_t sort_workspace_bytes(size_t n, bool pairs);

// Enqueue the whole sort of n items (1 <= n < 2^32) on `stream`, using the
// caller's workspace (at least layout_for(n, pairs).total bytes).
rs_status enqueue_sort(uint32_t* keys, uint32_t* vals, uint32_t n, cudaStream_t stream,
                       void* workspace, size_t workspace_bytes, uint32_t key_type = 0);

// Alg. 2's local MSD pass: one stable counting-sort pass of n (1 <= n <
// 2^32) keys (with values when vals != nullptr) by digit 3 from the inputs
// into the outputs, and the 257 bucket offsets; workspace as for a sort.
rs_status enqueue_msd_partition(const uint32_t* keys, const uint32_t* vals, uint32_t n,
                                uint32_t* out_keys, uint32_t* out_vals, uint32_t* bucket_off,
                                cudaStream_t stream, void* workspace, size_t workspace_bytes);

// The sort with 11-bit digits (three passes of 11, 11 and 10 bits;
// rs_digits11.cu): two alternate key (and value) buffers, per-chunk digit
// counts of at most kD11MaxChunks chunks, and the 2048 bucket totals.
constexpr uint32_t kD11MaxChunks = 1024;
struct Layout11 {
    size_t alt_keys[2], alt_vals[2], counts, totals, total;
    uint32_t max_chunks;
};
Layout11 layout11(size_t n, bool pairs);
int d11_shape_count();
rs_status enqueue_sort11(uint32_t* keys, uint32_t* vals, uint32_t n, cudaStream_t stream,
                         void* workspace, size_t workspace_bytes);

// Wide items: 64-bit keys (eight passes; key_type KEY_U64, KEY_I64 or
// KEY_F64) carrying no, 32-bit or 64-bit values (val_bytes 0, 4 or 8), and
// 32-bit keys (KEY_U32, KEY_I32, KEY_F32) carrying 64-bit values.  Every
// array size takes the scatter passes.
Layout layout_wide(size_t n, bool key64, uint32_t val_bytes);
rs_status enqueue_sort_wide(void* keys, void* vals, uint32_t n, uint32_t key_type,
                            uint32_t val_bytes, cudaStream_t stream, void* workspace,
                            size_t workspace_bytes);
// Scatter-pass tiles of the wide sorts: 384 threads, items per thread.
constexpr int kWideThreads = 384;
constexpr int kWideItems64 = 7;     // 64-bit keys, no or 32-bit values
constexpr int kWideItems64V64 = 6;  // 64-bit keys, 64-bit values
constexpr int kWideItems32V64 = 7;  // 32-bit keys, 64-bit values
// One scatter pass of 64-bit keys (rs_sort64.cu); wide = 64-bit status words.
rs_status launch_pass_k64(uint32_t key_type, uint32_t val_bytes, bool wide,
                          unsigned long long* ka, void* va, unsigned long long* kb, void* vb,
                          uint32_t n, uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status,
                          void* status_clear, cudaStream_t stream);

// Enqueue the digit histograms of n keys into hist[4 * 256] (zeroed first).
rs_status enqueue_histograms(const uint32_t* keys, uint32_t n, uint32_t* hist,
                             cudaStream_t stream);
// The same, added into hist (zeroed by the caller), counting the digits of
// the ordered words of typed keys, and clearing clear_bytes at `clear`.
rs_status enqueue_hist4(const uint32_t* keys, uint32_t n, uint32_t* hist, void* clear,
                        size_t clear_bytes, uint32_t key_type, cudaStream_t stream);

// Segmented scatter passes: per-tile geometry and per-segment bucket bases
// built on the device, and an upper bound of the tile count for the launch.
struct SegView {
    const uint4* tile_geo = nullptr;
    const uint32_t* gofs = nullptr;
    uint32_t max_tiles = 0;
};

// Scatter-pass launchers, one per value flavour (separate translation units);
// seg == nullptr for the unsegmented sort.
// key_type: KEY_U32, KEY_I32 or KEY_F32 (rs_device.cuh).
// slot: the plan entry of the launch (the pass, or MSD_SLOT).
rs_status launch_onesweep_keys(int cfg, bool wide, uint32_t* ka, uint32_t* kb, uint32_t n,
                               uint32_t pass, uint32_t slot, Ctrl* ctrl, uint32_t* sticky,
                               void* status, void* status_clear, const SegView* seg,
                               uint32_t key_type, cudaStream_t stream);
rs_status launch_onesweep_pairs(int cfg, bool wide, uint32_t* ka, uint32_t* va, uint32_t* kb,
                                uint32_t* vb, uint32_t n, uint32_t pass, uint32_t slot,
                                Ctrl* ctrl, uint32_t* sticky, void* status, void* status_clear,
                                const SegView* seg, uint32_t key_type, cudaStream_t stream);

// One-CTA sort in shared memory: of every small segment listed by the
// segmented planner (off != nullptr; none longer than max_items), or of the
// single array [0, single_n) with single_n <= max_items <= small_sort_capacity().
// bits: digit width, 4 or 8.
// src_keys / src_vals (default: keys / vals, in place) is where items are read.
rs_status launch_small_sort(uint32_t* keys, uint32_t* vals, const uint32_t* off,
                            const uint32_t* small_list, const Ctrl* ctrl, uint32_t single_n,
                            uint32_t max_items, int bits, uint32_t key_type, cudaStream_t stream,
                            const uint32_t* src_keys = nullptr,
                            const uint32_t* src_vals = nullptr);
uint32_t small_sort_capacity();

// One-warp sort in shared memory: of every tiny segment listed by the
// segmented planner (off != nullptr), or of the single array [0, single_n)
// with single_n <= warp_sort_capacity().  bits: digit width, 4 or 8.
rs_status launch_warp_sort(uint32_t* keys, uint32_t* vals, const uint32_t* off,
                           const uint32_t* tiny_list, const Ctrl* ctrl, uint32_t single_n,
                           int bits, uint32_t key_type, cudaStream_t stream,
                           const uint32_t* src_keys = nullptr, const uint32_t* src_vals = nullptr);
uint32_t warp_sort_capacity();

// Workspace layout of a segmented sort of n items in num_segments segments.
struct SegLayout {
    size_t ctrl, status0, status1, alt_keys, alt_vals, tile_geo, tiny_list, small_list, large_first,
        gofs, total;
    uint32_t max_tiles, max_large;
};
SegLayout seg_layout_for(size_t n, bool pairs, uint32_t num_segments);
// Segmented sorts of wide items (64-bit keys, or 32-bit keys with 64-bit
// values; rs_segmented_wide.cu).
SegLayout seg_layout_wide(size_t n, bool key64, uint32_t val_bytes, uint32_t num_segments);
rs_status enqueue_sort_segmented_wide(void* keys, void* vals, uint32_t n,
                                      const uint32_t* offsets, uint32_t num_segments,
                                      uint32_t key_type, uint32_t val_bytes, cudaStream_t stream,
                                      void* workspace, size_t workspace_bytes);
rs_status enqueue_sort_segmented(uint32_t* keys, uint32_t* vals, uint32_t n,
                                 const uint32_t* offsets, uint32_t num_segments,
                                 cudaStream_t stream, void* workspace, size_t workspace_bytes,
                                 uint32_t key_type = 0);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Launch `kern` on `stream`; with knobs().pdl set, as a programmatic
// dependent of the kernel before it on the stream, so that it becomes
// resident while that kernel finishes (the kernel calls pdl_wait() before
// reading that kernel's output).
template <typename... Params, typename... Args>
cudaError_t launch_after_previous(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t stream, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = knobs().pdl ? 1u : 0u;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// One bit per device (ordinal < 64) for one-time host setup of a kernel
// (its shared-memory limit), safe when several host threads enqueue sorts.
struct DeviceOnce {
    std::atomic<uint64_t> bits{0};
    bool done(int dev) const { return (bits.load(std::memory_order_acquire) >> dev) & 1u; }
    void mark(int dev) { bits.fetch_or(uint64_t(1) << dev, std::memory_order_release); }
};

// Raise the dynamic shared-memory limit of `kern` to `bytes` once per device.
template <typename Kern>
rs_status allow_smem_once(Kern kern, size_t bytes, DeviceOnce& once) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RS_ERR_CUDA;
    if (!once.done(dev)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess)
            return RS_ERR_CUDA;
        once.mark(dev);
    }
    return RS_OK;
}

}  // namespace rs
