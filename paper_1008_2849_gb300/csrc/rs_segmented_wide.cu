// rs_segmented_wide.cu -- host side of the segmented sort of wide items:
// 64-bit keys (eight passes) with no, 32-bit or 64-bit values, and 32-bit
// keys with 64-bit values (four passes); unsigned or typed keys.  Segments
// of up to kWideWarpMax items are sorted by one warp each in shared memory;
// every longer segment takes the segmented scatter passes.
#include "rs_internal.h"
#include "rs_onesweep_launch.cuh"
#include "rs_segmented.cuh"
#include "rs_segmented_wide.cuh"

namespace rs {

namespace {

constexpr int kWideWarpItems = 8;                             // one warp: up to 256 items
constexpr uint32_t kWideWarpMax = 32u * kWideWarpItems;
constexpr int B_SEG = 2, W_SEG = 8;

uint32_t wide_items(bool key64, uint32_t val_bytes) {
    return key64 ? (val_bytes == 8 ? kWideItems64V64 : kWideItems64) : kWideItems32V64;
}

// One scatter pass over the large segments' tiles, both instances for typed
// keys (the passes that need no maps run without them).
template <typename K, typename V, bool PAIRS>
rs_status seg_pass(uint32_t key_type, K* ka, V* va, K* kb, V* vb, uint32_t n, uint32_t pass,
                   Ctrl* ctrl, uint32_t* sticky, void* status, void* status_clear,
                   const SegView& view, cudaStream_t stream) {
    constexpr int J = sizeof(K) == 8 ? (PAIRS && sizeof(V) == 8 ? kWideItems64V64 : kWideItems64)
                                     : kWideItems32V64;
    const bool plain = key_type == KEY_U32 || key_type == KEY_U64;
    if (!plain && !typed_split(n))  // small sorts: the mapping instance runs every pass
        return launch_onesweep_shape<kWideThreads, J, B_SEG, W_SEG, PAIRS, uint32_t, true, true, K,
                                     V>(ka, va, kb, vb, n, pass, pass, ctrl, sticky, status,
                                        status_clear, view, key_type, stream);
    if (plain)
        return launch_onesweep_shape<kWideThreads, J, B_SEG, W_SEG, PAIRS, uint32_t, true, false, K,
                                     V>(ka, va, kb, vb, n, pass, pass, ctrl, sticky, status,
                                        status_clear, view, KEY_U32, stream);
    const rs_status st =
        launch_onesweep_shape<kWideThreads, J, B_SEG, W_SEG, PAIRS, uint32_t, true, false, K, V>(
            ka, va, kb, vb, n, pass, pass, ctrl, sticky, status, status_clear, view,
            key_type | ROLE_PLAIN_PASSES, stream);
    if (st != RS_OK) return st;
    return launch_onesweep_shape<kWideThreads, J, B_SEG, W_SEG, PAIRS, uint32_t, true, true, K, V>(
        ka, va, kb, vb, n, pass, pass, ctrl, sticky, status, status_clear, view,
        key_type | ROLE_MAP_PASSES, stream);
}

template <typename K, typename V, bool PAIRS>
rs_status warp_sort(K* keys, V* vals, const uint32_t* off, const uint32_t* tiny_list,
                    const Ctrl* ctrl, uint32_t key_type, int sm_count, cudaStream_t stream) {
    using L = WideWarpSmem<K, V, PAIRS, kWideWarpItems>;
    auto kern = k_warp_sort_wide<K, V, PAIRS, kWideWarpItems>;
    static DeviceOnce smem_set;
    rs_status st = allow_smem_once(kern, L::BYTES, smem_set);
    if (st != RS_OK) return st;
    note_launch_begin(KK_WARP, stream);
    kern<<<sm_count * 4, WIDE_WARP_THREADS, L::BYTES, stream>>>(keys, vals, off, tiny_list, ctrl,
                                                               key_type);
    note_launch_end(KK_WARP, stream);
    return cudaPeekAtLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

// The whole sequence for one combination of key and value widths.
template <typename K, typename V, bool PAIRS>
rs_status run(K* keys, V* vals, uint32_t n, const uint32_t* offsets, uint32_t num_segments,
              uint32_t key_type, cudaStream_t stream, void* workspace, const SegLayout& L) {
    constexpr uint32_t NP = sizeof(K) == 8 ? PASSES64 : PASSES;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    char* ws = static_cast<char*>(workspace);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
    void* status[2] = {ws + L.status0, ws + L.status1};
    K* alt_k = reinterpret_cast<K*>(ws + L.alt_keys);
    V* alt_v = PAIRS ? reinterpret_cast<V*>(ws + L.alt_vals) : nullptr;
    uint4* tile_geo = reinterpret_cast<uint4*>(ws + L.tile_geo);
    uint32_t* tiny_list = reinterpret_cast<uint32_t*>(ws + L.tiny_list);
    uint32_t* small_list = reinterpret_cast<uint32_t*>(ws + L.small_list);
    uint32_t* large_first = reinterpret_cast<uint32_t*>(ws + L.large_first);
    uint32_t* gofs = reinterpret_cast<uint32_t*>(ws + L.gofs);
    const uint32_t tile = (uint32_t)kWideThreads * wide_items(sizeof(K) == 8, PAIRS ? sizeof(V) : 0);
    const size_t status_vec4 = (L.status1 - L.status0) / sizeof(uint4);

    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return RS_ERR_CUDA;
    if (L.max_large > 0 &&
        cudaMemsetAsync(gofs, 0, (size_t)L.max_large * NP * RADIX * 4, stream) != cudaSuccess)
        return RS_ERR_CUDA;
    // Segments of up to kWideWarpMax items: one warp each; every longer one
    // is large (no one-CTA class for wide items).
    note_launch_begin(KK_SEG_PLAN, stream);
    k_seg_plan<<<1, 1024, 0, stream>>>(offsets, num_segments, n, tile, kWideWarpMax, kWideWarpMax,
                                       ctrl, di.sticky, tile_geo, tiny_list, small_list,
                                       large_first, NP);
    note_launch_end(KK_SEG_PLAN, stream);
    if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;
    st = warp_sort<K, V, PAIRS>(keys, vals, offsets, tiny_list, ctrl, key_type, di.sm_count, stream);
    if (st != RS_OK) return st;

    note_launch_begin(KK_SEG_HIST, stream);
    if constexpr (sizeof(K) == 8) {
        auto kern = key_type == KEY_U64 ? k_seg_hist64<false> : k_seg_hist64<true>;
        kern<<<di.sm_count, SEG_HIST64_THREADS, 0, stream>>>(
            keys, ctrl, tile_geo, gofs, static_cast<uint4*>(status[0]), (uint32_t)status_vec4,
            key_type);
    } else {
        constexpr size_t SMEM = SEG_HIST_COL_WORDS * sizeof(uint32_t);
        auto kern = key_type != KEY_U32 ? k_seg_hist<true> : k_seg_hist<false>;
        static DeviceOnce smem_set[2];
        st = allow_smem_once(kern, SMEM, smem_set[key_type != KEY_U32 ? 1 : 0]);
        if (st != RS_OK) return st;
        kern<<<di.sm_count, SEG_HIST_THREADS, SMEM, stream>>>(
            keys, ctrl, tile_geo, gofs, static_cast<uint4*>(status[0]), (uint32_t)status_vec4,
            key_type);
    }
    note_launch_end(KK_SEG_HIST, stream);
    note_launch_begin(KK_SEG_SCAN, stream);
    k_seg_scan<NP><<<di.sm_count * 2, 1024, 0, stream>>>(ctrl, gofs, large_first);
    note_launch_end(KK_SEG_SCAN, stream);
    if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;

    SegView view;
    view.tile_geo = tile_geo;
    view.gofs = gofs;
    view.max_tiles = L.max_tiles;
    for (uint32_t p = 0; p < NP; ++p) {
        void* cur = status[p & 1];
        void* next = p + 1 < NP ? status[(p + 1) & 1] : nullptr;
        st = seg_pass<K, V, PAIRS>(key_type, keys, vals, alt_k, alt_v, n, p, ctrl, di.sticky, cur,
                                   next, view, stream);
        if (st != RS_OK) return st;
    }
    return RS_OK;
}

}  // namespace

SegLayout seg_layout_wide(size_t n, bool key64, uint32_t val_bytes, uint32_t num_segments) {
    SegLayout L{};
    const size_t tile = (size_t)kWideThreads * wide_items(key64, val_bytes);
    const size_t large = std::min<size_t>(num_segments, n / (kWideWarpMax + 1) + 1);
    const uint32_t np = key64 ? PASSES64 : PASSES;
    L.max_large = (uint32_t)large;
    L.max_tiles = (uint32_t)((n + tile - 1) / tile + large);
    const size_t status_bytes = (size_t)L.max_tiles * RADIX * 4;
    size_t off = 0;
    L.ctrl = off;
    off = align_up(off + sizeof(Ctrl), 256);
    L.status0 = off;
    off = align_up(off + status_bytes, 256);
    L.status1 = off;
    off = align_up(off + status_bytes, 256);
    L.alt_keys = off;
    off = align_up(off + n * (key64 ? 8 : 4), 256);
    L.alt_vals = off;
    off = align_up(off + n * val_bytes, 256);
    L.tile_geo = off;
    off = align_up(off + (size_t)L.max_tiles * 16, 256);
    L.tiny_list = off;
    off = align_up(off + (size_t)num_segments * 4, 256);
    L.small_list = off;
    off = align_up(off + (size_t)num_segments * 4, 256);
    L.large_first = off;
    off = align_up(off + large * 4, 256);
    L.gofs = off;
    off = align_up(off + large * np * RADIX * 4, 256);
    L.total = off;
    return L;
}

rs_status enqueue_sort_segmented_wide(void* keys, void* vals, uint32_t n,
                                      const uint32_t* offsets, uint32_t num_segments,
                                      uint32_t key_type, uint32_t val_bytes, cudaStream_t stream,
                                      void* workspace, size_t workspace_bytes) {
    if (key_type > KEY_F64 || (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) ||
        (val_bytes == 0) != (vals == nullptr))
        return RS_ERR_INVALID_ARG;
    const bool key64 = key_type >= KEY_U64;
    if (!key64 && val_bytes != 8) return RS_ERR_INVALID_ARG;  // the 32-bit sorts serve these
    const SegLayout L = seg_layout_wide(n, key64, val_bytes, num_segments);
    if (workspace == nullptr || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    using u64 = unsigned long long;
    if (!key64)
        return run<uint32_t, u64, true>(static_cast<uint32_t*>(keys), static_cast<u64*>(vals), n,
                                        offsets, num_segments, key_type, stream, workspace, L);
    switch (val_bytes) {
    case 0:
        return run<u64, uint32_t, false>(static_cast<u64*>(keys), nullptr, n, offsets,
                                         num_segments, key_type, stream, workspace, L);
    case 4:
        return run<u64, uint32_t, true>(static_cast<u64*>(keys), static_cast<uint32_t*>(vals), n,
                                        offsets, num_segments, key_type, stream, workspace, L);
    default:
        return run<u64, u64, true>(static_cast<u64*>(keys), static_cast<u64*>(vals), n, offsets,
                                   num_segments, key_type, stream, workspace, L);
    }
}

}  // namespace rs
