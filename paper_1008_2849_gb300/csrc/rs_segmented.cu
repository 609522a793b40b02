// rs_segmented.cu -- host side of the segmented sort: workspace layout and
// launch sequence.
#include "rs_internal.h"
#include "rs_segmented.cuh"

namespace rs {

namespace {

constexpr uint32_t kMinLargeSegment = 4097;  // segments up to 4096 items always take the one-CTA sort

}  // namespace

SegLayout seg_layout_for(size_t n, bool pairs, uint32_t num_segments) {
    SegLayout L{};
    const size_t tile = (size_t)smallest_tile();
    const size_t large = std::min<size_t>(num_segments, n / kMinLargeSegment + 1);
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
    off = align_up(off + n * 4, 256);
    L.alt_vals = off;
    if (pairs) off = align_up(off + n * 4, 256);
    L.tile_geo = off;
    off = align_up(off + (size_t)L.max_tiles * 16, 256);
    L.tiny_list = off;
    off = align_up(off + (size_t)num_segments * 4, 256);
    L.small_list = off;
    off = align_up(off + (size_t)num_segments * 4, 256);
    L.large_first = off;
    off = align_up(off + large * 4, 256);
    L.gofs = off;
    off = align_up(off + large * PASSES * RADIX * 4, 256);
    L.total = off;
    return L;
}

rs_status enqueue_sort_segmented(uint32_t* keys, uint32_t* vals, uint32_t n,
                                 const uint32_t* offsets, uint32_t num_segments,
                                 cudaStream_t stream, void* workspace, size_t workspace_bytes,
                                 uint32_t key_type) {
    if (key_type > KEY_F32) return RS_ERR_INVALID_ARG;
    const bool pairs = vals != nullptr;
    const SegLayout L = seg_layout_for(n, pairs, num_segments);
    if (workspace == nullptr || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    char* ws = static_cast<char*>(workspace);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
    void* status[2] = {ws + L.status0, ws + L.status1};
    uint32_t* alt_k = reinterpret_cast<uint32_t*>(ws + L.alt_keys);
    uint32_t* alt_v = pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals) : nullptr;
    uint4* tile_geo = reinterpret_cast<uint4*>(ws + L.tile_geo);
    uint32_t* tiny_list = reinterpret_cast<uint32_t*>(ws + L.tiny_list);
    uint32_t* small_list = reinterpret_cast<uint32_t*>(ws + L.small_list);
    uint32_t* large_first = reinterpret_cast<uint32_t*>(ws + L.large_first);
    uint32_t* gofs = reinterpret_cast<uint32_t*>(ws + L.gofs);

    const ClassKnobs& ck = knobs().cls[size_class(n / num_segments)];
    const int cfg = key_type != KEY_U32 ? kTypedShape : ck.tile_seg;
    const uint32_t tile = (uint32_t)(kTileConfigs[cfg].threads * kTileConfigs[cfg].items);
    uint32_t small_max = (uint32_t)ck.small_max;
    if (small_max < kMinLargeSegment - 1) small_max = kMinLargeSegment - 1;
    if (small_max > small_sort_capacity()) small_max = small_sort_capacity();
    uint32_t warp_max = (uint32_t)ck.warp_max;
    if (warp_max > warp_sort_capacity()) warp_max = warp_sort_capacity();

    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return RS_ERR_CUDA;
    if (L.max_large > 0 &&
        cudaMemsetAsync(gofs, 0, (size_t)L.max_large * PASSES * RADIX * 4, stream) != cudaSuccess)
        return RS_ERR_CUDA;
    note_launch_begin(KK_SEG_PLAN, stream);
    k_seg_plan<<<1, 1024, 0, stream>>>(offsets, num_segments, n, tile, warp_max, small_max, ctrl,
                                       di.sticky, tile_geo, tiny_list, small_list, large_first);
    note_launch_end(KK_SEG_PLAN, stream);
    if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;

    // Tiny and small segments: independent of the large ones (disjoint ranges).
    if (warp_max >= 2) {
        st = launch_warp_sort(keys, vals, offsets, tiny_list, ctrl, 0, ck.small_bits, key_type,
                              stream);
        if (st != RS_OK) return st;
    }
    st = launch_small_sort(keys, vals, offsets, small_list, ctrl, 0, small_max, ck.small_bits,
                           key_type, stream);
    if (st != RS_OK) return st;

    // Large segments: histograms, bucket bases, four scatter passes.
    note_launch_begin(KK_SEG_HIST, stream);
    {
        constexpr size_t SMEM = SEG_HIST_COL_WORDS * sizeof(uint32_t);
        auto kern = key_type != KEY_U32 ? k_seg_hist<true> : k_seg_hist<false>;
        static DeviceOnce smem_set[2];
        st = allow_smem_once(kern, SMEM, smem_set[key_type != KEY_U32 ? 1 : 0]);
        if (st != RS_OK) return st;
        if (launch_after_previous(kern, dim3(di.sm_count), dim3(SEG_HIST_THREADS), SMEM, stream,
                                  (const uint32_t*)keys, (const Ctrl*)ctrl,
                                  (const uint4*)tile_geo, gofs, static_cast<uint4*>(status[0]),
                                  (uint32_t)((L.status1 - L.status0) / sizeof(uint4)),
                                  key_type) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    note_launch_end(KK_SEG_HIST, stream);
    note_launch_begin(KK_SEG_SCAN, stream);
    const cudaError_t se = launch_after_previous(k_seg_scan<PASSES>, dim3(di.sm_count * 2),
                                                 dim3(1024), 0, stream, (const Ctrl*)ctrl, gofs,
                                                 (const uint32_t*)large_first);
    note_launch_end(KK_SEG_SCAN, stream);
    if (se != cudaSuccess) return RS_ERR_CUDA;

    SegView view;
    view.tile_geo = tile_geo;
    view.max_tiles = L.max_tiles;
    for (uint32_t p = 0; p < PASSES; ++p) {
        view.gofs = gofs;
        void* cur = status[p & 1];
        void* next = p + 1 < PASSES ? status[(p + 1) & 1] : nullptr;
        st = pairs ? launch_onesweep_pairs(cfg, false, keys, vals, alt_k, alt_v, n, p, p, ctrl,
                                           di.sticky, cur, next, &view, key_type, stream)
                   : launch_onesweep_keys(cfg, false, keys, alt_k, n, p, p, ctrl, di.sticky, cur,
                                          next, &view, key_type, stream);
        if (st != RS_OK) return st;
    }
    return RS_OK;
}

}  // namespace rs
