// rs_onesweep_launch.cuh -- host launcher of k_onesweep for every tile shape
// of kTileConfigs; included once per value flavour (keys / pairs).
#pragma once

#include "rs_internal.h"
#include "rs_onesweep.cuh"

namespace rs {

// Compile-time parameters of tile shape I of RS_TILE_SHAPES.
template <int I> struct TileShape;
#define RS_SHAPE_STRUCT(I, T, J, B, W)                                                    \
    template <> struct TileShape<I> {                                                     \
        static constexpr int threads = T, items = J, min_blocks = B, window = W;          \
    };
RS_TILE_SHAPES(RS_SHAPE_STRUCT)
#undef RS_SHAPE_STRUCT

template <int THREADS, int ITEMS, int MIN_BLOCKS, int WINDOW, bool PAIRS, typename S, bool SEG,
          bool TYPED, typename K = uint32_t, typename V = uint32_t>
static rs_status launch_onesweep_shape(K* ka, V* va, K* kb, V* vb,
                                       uint32_t n, uint32_t pass, uint32_t slot, Ctrl* ctrl,
                                       uint32_t* sticky,
                                       void* status, void* status_clear, const SegView& seg,
                                       uint32_t key_type, cudaStream_t stream) {
    using L = OnesweepSmem<THREADS, ITEMS, PAIRS, (int)(sizeof(K) / 4), (int)(sizeof(V) / 4)>;
    constexpr uint32_t TILE = L::TILE;
    auto kern = k_onesweep<THREADS, ITEMS, MIN_BLOCKS, PAIRS, S, WINDOW, SEG, TYPED, K, V>;
    static std::atomic<int> ctas_per_sm[64];  // per device: resident CTAs per SM (0: unknown)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RS_ERR_CUDA;
    int resident = ctas_per_sm[dev].load(std::memory_order_acquire);
    if (resident == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES) !=
            cudaSuccess)
            return RS_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, THREADS, L::BYTES) !=
                cudaSuccess ||
            resident < 1)
            return RS_ERR_CUDA;
        ctas_per_sm[dev].store(resident, std::memory_order_release);
    }
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    // Segmented: the tile count is only known on the device (ctrl->seg_tiles).
    const uint32_t tiles = SEG ? seg.max_tiles : (uint32_t)((n + (size_t)TILE - 1) / TILE);
    uint32_t grid = (uint32_t)(di.sm_count * resident);
    if (grid > tiles) grid = tiles;
    if (grid == 0) return RS_OK;
    note_launch_begin(SEG ? KK_SEG_ONESWEEP : KK_ONESWEEP, stream);
    const cudaError_t e = launch_after_previous(
        kern, dim3(grid), dim3(THREADS), L::BYTES, stream, ka, va, kb, vb, n, pass, slot, tiles,
        ctrl, sticky, static_cast<S*>(status), static_cast<S*>(status_clear), tiles * RADIX,
        knobs().spin_limit, knobs().debug, seg.tile_geo, seg.gofs, key_type);
    note_launch_end(SEG ? KK_SEG_ONESWEEP : KK_ONESWEEP, stream);
    return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

template <bool PAIRS, typename S, bool SEG>
static rs_status launch_onesweep_variant(int cfg, uint32_t* ka, uint32_t* va, uint32_t* kb,
                                         uint32_t* vb, uint32_t n, uint32_t pass, uint32_t slot,
                                         Ctrl* ctrl,
                                         uint32_t* sticky, void* status, void* status_clear,
                                         const SegView& seg, uint32_t key_type,
                                         cudaStream_t stream) {
    if (key_type != KEY_U32) {
        // Typed keys: from typed_split_min items on, the passes that need no
        // maps run without them (see ROLE_PLAIN_PASSES) and both instances
        // are launched for every pass; below it the mapping instance alone
        // runs every pass, mapping where the plan needs it.
        using T = TileShape<kTypedShape>;
        if (!typed_split(n))
            return launch_onesweep_shape<T::threads, T::items, T::min_blocks, T::window, PAIRS, S,
                                         SEG, true>(ka, va, kb, vb, n, pass, slot, ctrl, sticky,
                                                    status, status_clear, seg, key_type, stream);
        const rs_status st =
            launch_onesweep_shape<T::threads, T::items, T::min_blocks, T::window, PAIRS, S, SEG,
                                  false>(ka, va, kb, vb, n, pass, slot, ctrl, sticky, status,
                                         status_clear, seg, key_type | ROLE_PLAIN_PASSES, stream);
        if (st != RS_OK) return st;
        return launch_onesweep_shape<T::threads, T::items, T::min_blocks, T::window, PAIRS, S, SEG,
                                     true>(ka, va, kb, vb, n, pass, slot, ctrl, sticky, status,
                                           status_clear, seg, key_type | ROLE_MAP_PASSES, stream);
    }
    switch (cfg) {
#define RS_CASE(I, T, J, B, W)                                                                    \
    case I:                                                                                       \
        return launch_onesweep_shape<T, J, B, W, PAIRS, S, SEG, false>(                           \
            ka, va, kb, vb, n, pass, slot, ctrl, sticky, status, status_clear, seg, KEY_U32, stream);
        RS_TILE_SHAPES(RS_CASE)
#undef RS_CASE
    default: return RS_ERR_INVALID_ARG;
    }
}

}  // namespace rs
