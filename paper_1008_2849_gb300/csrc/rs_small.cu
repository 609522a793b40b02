// rs_small.cu -- host launchers of the on-chip sorts (rs_small.cuh): the
// one-warp sort and the one-CTA sort, each at digit width 4 or 8.
#include "rs_internal.h"
#include "rs_small.cuh"

namespace rs {

namespace {

// One-CTA sort shapes: 256 threads x 16 items (4096) and 512 x 16 (8192).
template <int THREADS, int ITEMS, int BITS, bool PAIRS>
rs_status launch_small_shape(uint32_t* keys, uint32_t* vals, const uint32_t* src_keys,
                             const uint32_t* src_vals, const uint32_t* off,
                             const uint32_t* list, const Ctrl* ctrl, uint32_t single_n,
                             uint32_t grid, uint32_t key_type, cudaStream_t stream) {
    constexpr uint32_t CAP = THREADS * ITEMS;
    constexpr size_t SMEM =
        ((PAIRS ? 4u : 2u) * CAP + (THREADS / 32) * (1u << BITS)) * sizeof(uint32_t);
    auto kern = k_small_sort<THREADS, ITEMS, BITS, PAIRS>;
    static DeviceOnce smem_set;
    rs_status st = allow_smem_once(kern, SMEM, smem_set);
    if (st != RS_OK) return st;
    note_launch_begin(KK_SMALL, stream);
    const cudaError_t e = launch_after_previous(kern, dim3(grid), dim3(THREADS), SMEM, stream, keys,
                                                vals, src_keys, src_vals, off, list, ctrl,
                                                single_n, key_type);
    note_launch_end(KK_SMALL, stream);
    return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

template <int BITS, bool PAIRS>
rs_status launch_small_bits(uint32_t* keys, uint32_t* vals, const uint32_t* src_keys,
                            const uint32_t* src_vals, const uint32_t* off,
                            const uint32_t* list, const Ctrl* ctrl, uint32_t single_n,
                            uint32_t max_items, uint32_t grid, uint32_t key_type,
                            cudaStream_t stream) {
    if (max_items <= 4096)
        return launch_small_shape<256, 16, BITS, PAIRS>(keys, vals, src_keys, src_vals, off, list,
                                                        ctrl, single_n, grid, key_type, stream);
    return launch_small_shape<512, 16, BITS, PAIRS>(keys, vals, src_keys, src_vals, off, list, ctrl,
                                                    single_n, grid, key_type, stream);
}

template <int BITS, bool PAIRS>
rs_status launch_warp_bits(uint32_t* keys, uint32_t* vals, const uint32_t* src_keys,
                           const uint32_t* src_vals, const uint32_t* off,
                           const uint32_t* list, const Ctrl* ctrl, uint32_t single_n,
                           uint32_t grid, uint32_t key_type, cudaStream_t stream) {
    using L = WarpSortSmem<WARP_SORT_ITEMS, BITS, PAIRS>;
    auto kern = k_warp_sort<WARP_SORT_ITEMS, BITS, PAIRS>;
    static DeviceOnce smem_set;
    rs_status st = allow_smem_once(kern, L::BYTES, smem_set);
    if (st != RS_OK) return st;
    note_launch_begin(KK_WARP, stream);
    const cudaError_t e =
        launch_after_previous(kern, dim3(grid), dim3(WARP_SORT_THREADS), L::BYTES, stream, keys,
                              vals, src_keys, src_vals, off, list, ctrl, single_n, key_type);
    note_launch_end(KK_WARP, stream);
    return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

}  // namespace

uint32_t small_sort_capacity() { return 8192; }
uint32_t warp_sort_capacity() { return 32 * WARP_SORT_ITEMS; }

rs_status launch_small_sort(uint32_t* keys, uint32_t* vals, const uint32_t* off,
                            const uint32_t* small_list, const Ctrl* ctrl, uint32_t single_n,
                            uint32_t max_items, int bits, uint32_t key_type, cudaStream_t stream,
                            const uint32_t* src_keys, const uint32_t* src_vals) {
    if (max_items > small_sort_capacity()) return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    // Single array: one CTA.  Segment list: a grid-stride loop over it.
    const uint32_t grid = off == nullptr ? 1u : (uint32_t)di.sm_count * 4u;
    const bool pairs = vals != nullptr;
    const uint32_t* sk = src_keys ? src_keys : keys;
    const uint32_t* sv = src_keys ? src_vals : vals;
    if (bits == 4)
        return pairs ? launch_small_bits<4, true>(keys, vals, sk, sv, off, small_list, ctrl,
                                                  single_n, max_items, grid, key_type, stream)
                     : launch_small_bits<4, false>(keys, vals, sk, sv, off, small_list, ctrl,
                                                   single_n, max_items, grid, key_type, stream);
    return pairs ? launch_small_bits<8, true>(keys, vals, sk, sv, off, small_list, ctrl, single_n,
                                              max_items, grid, key_type, stream)
                 : launch_small_bits<8, false>(keys, vals, sk, sv, off, small_list, ctrl, single_n,
                                               max_items, grid, key_type, stream);
}

rs_status launch_warp_sort(uint32_t* keys, uint32_t* vals, const uint32_t* off,
                           const uint32_t* tiny_list, const Ctrl* ctrl, uint32_t single_n,
                           int bits, uint32_t key_type, cudaStream_t stream,
                           const uint32_t* src_keys, const uint32_t* src_vals) {
    if (off == nullptr && single_n > warp_sort_capacity()) return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    const uint32_t grid = off == nullptr ? 1u : (uint32_t)di.sm_count * 3u;
    const bool pairs = vals != nullptr;
    const uint32_t* sk = src_keys ? src_keys : keys;
    const uint32_t* sv = src_keys ? src_vals : vals;
    if (bits == 4)
        return pairs ? launch_warp_bits<4, true>(keys, vals, sk, sv, off, tiny_list, ctrl, single_n,
                                                 grid, key_type, stream)
                     : launch_warp_bits<4, false>(keys, vals, sk, sv, off, tiny_list, ctrl,
                                                  single_n, grid, key_type, stream);
    return pairs ? launch_warp_bits<8, true>(keys, vals, sk, sv, off, tiny_list, ctrl, single_n,
                                             grid, key_type, stream)
                 : launch_warp_bits<8, false>(keys, vals, sk, sv, off, tiny_list, ctrl, single_n,
                                              grid, key_type, stream);
}

}  // namespace rs
