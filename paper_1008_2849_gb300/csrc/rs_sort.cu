// rs_sort.cu -- histogram and plan kernels, workspace layout and the
// enqueue sequence of one unsegmented sort.
#include "rs_internal.h"
#include "rs_hist_plan.cuh"

namespace rs {

// Must list the shapes of RS_TILE_SHAPES (rs_onesweep_launch.cuh) in order.
#define RS_SHAPE_ENTRY(I, T, J, B, W) {T, J, B, W},
const TileConfig kTileConfigs[NUM_TILE_CONFIGS] = {RS_TILE_SHAPES(RS_SHAPE_ENTRY)};
#undef RS_SHAPE_ENTRY

int smallest_tile() {
    int t = kTileConfigs[0].threads * kTileConfigs[0].items;
    for (int i = 1; i < NUM_TILE_CONFIGS; ++i)
        if (kTileConfigs[i].threads * kTileConfigs[i].items < t)
            t = kTileConfigs[i].threads * kTileConfigs[i].items;
    return t;
}

constexpr int HIST_THREADS = 512;

Layout layout_for(size_t n, bool pairs) {
    Layout L{};
    const size_t tile = (size_t)smallest_tile();
    L.tiles = (uint32_t)((n + tile - 1) / tile);
    L.wide_status = n >= (size_t(1) << 30);
    const size_t status_bytes = (size_t)L.tiles * RADIX * (L.wide_status ? 8 : 4);
    size_t off = 0;
    L.ctrl = off;
    off = align_up(off + sizeof(Ctrl), 256);
    L.status0 = off;
    off = align_up(off + status_bytes, 256);
    L.status1 = off;
    off = align_up(off + status_bytes, 256);
    L.alt_keys = off;
    off = align_up(off + n * sizeof(uint32_t), 256);
    L.alt_vals = off;
    if (pairs) off = align_up(off + n * sizeof(uint32_t), 256);
    L.msd_off = off;  // MSD-first order: bucket offsets and bucket lists
    off = align_up(off + (RADIX + 1) * sizeof(uint32_t), 256);
    L.msd_tiny = off;
    off = align_up(off + RADIX * sizeof(uint32_t), 256);
    L.msd_small = off;
    off = align_up(off + RADIX * sizeof(uint32_t), 256);
    L.total = off;
    return L;
}

rs_status enqueue_hist4(const uint32_t* keys, uint32_t n, uint32_t* hist, void* clear,
                        size_t clear_bytes, uint32_t key_type, cudaStream_t stream) {
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    const uint32_t vec4 = (uint32_t)(n / 4);
    uint32_t blocks = (uint32_t)(di.sm_count * knobs().hist_ctas_per_sm);
    const uint32_t needed = (vec4 + 63) / 64 / (HIST_THREADS / 32) + 1;  // 64 vectors per warp
    if (blocks > needed) blocks = needed;
    if (blocks < 1) blocks = 1;
    if (knobs().hist_mode == HIST_COLUMNS) {
        constexpr int T = 1024;
        constexpr size_t SMEM = HIST_COL_WORDS * sizeof(uint32_t);
        auto kern = key_type != KEY_U32 ? k_hist4_cols<T, true> : k_hist4_cols<T, false>;
        static DeviceOnce smem_set[2];  // per instance
        st = allow_smem_once(kern, SMEM, smem_set[key_type != KEY_U32 ? 1 : 0]);
        if (st != RS_OK) return st;
        uint32_t grid = (uint32_t)di.sm_count;
        const uint32_t need = (vec4 + T - 1) / T;
        if (grid > need) grid = need > 0 ? need : 1;
        note_launch_begin(KK_HIST, stream);
        kern<<<grid, T, SMEM, stream>>>(keys, n, hist, static_cast<uint4*>(clear),
                                         (uint32_t)(clear_bytes / sizeof(uint4)), key_type);
        note_launch_end(KK_HIST, stream);
        return cudaPeekAtLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
    }
    const bool typed = key_type != KEY_U32;
    auto kern = typed ? k_hist4<HIST_THREADS, HIST_LEADER, true>
                      : k_hist4<HIST_THREADS, HIST_LEADER, false>;
    switch (knobs().hist_mode) {
    case HIST_ATOMIC:
        kern = typed ? k_hist4<HIST_THREADS, HIST_ATOMIC, true>
                     : k_hist4<HIST_THREADS, HIST_ATOMIC, false>;
        break;
    case HIST_MATCH:
        kern = typed ? k_hist4<HIST_THREADS, HIST_MATCH, true>
                     : k_hist4<HIST_THREADS, HIST_MATCH, false>;
        break;
    default: break;
    }
    note_launch_begin(KK_HIST, stream);
    kern<<<blocks, HIST_THREADS, 0, stream>>>(keys, n, hist, static_cast<uint4*>(clear),
                                              (uint32_t)(clear_bytes / sizeof(uint4)), key_type);
    note_launch_end(KK_HIST, stream);
    return cudaPeekAtLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

rs_status enqueue_histograms(const uint32_t* keys, uint32_t n, uint32_t* hist,
                             cudaStream_t stream) {
    if (cudaMemsetAsync(hist, 0, PASSES * RADIX * sizeof(uint32_t), stream) != cudaSuccess)
        return RS_ERR_CUDA;
    return enqueue_hist4(keys, n, hist, nullptr, 0, KEY_U32, stream);
}

rs_status enqueue_msd_partition(const uint32_t* keys, const uint32_t* vals, uint32_t n,
                                uint32_t* out_keys, uint32_t* out_vals, uint32_t* bucket_off,
                                cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    const bool pairs = vals != nullptr;
    const Layout L = layout_for(n, pairs);
    if (workspace == nullptr || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    char* ws = static_cast<char*>(workspace);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
    void* status = ws + L.status0;
    const size_t status_bytes = L.status1 - L.status0;
    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return RS_ERR_CUDA;
    st = enqueue_hist4(keys, n, &ctrl->hist[0][0], status, status_bytes, KEY_U32, stream);
    if (st != RS_OK) return st;
    note_launch_begin(KK_PLAN, stream);
    k_msd_plan<<<1, RADIX, 0, stream>>>(ctrl, n, bucket_off);
    note_launch_end(KK_PLAN, stream);
    if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;
    const ClassKnobs& ck = knobs().cls[size_class(n)];
    // The scatter kernels read the source through the plan's direction
    // (A -> B) and never write it.
    uint32_t* src_k = const_cast<uint32_t*>(keys);
    uint32_t* src_v = const_cast<uint32_t*>(vals);
    return pairs ? launch_onesweep_pairs(ck.tile_pairs, L.wide_status, src_k, src_v, out_keys,
                                         out_vals, n, PASSES - 1, MSD_SLOT, ctrl, di.sticky,
                                         status, nullptr, nullptr, KEY_U32, stream)
                 : launch_onesweep_keys(ck.tile_keys, L.wide_status, src_k, out_keys, n,
                                        PASSES - 1, MSD_SLOT, ctrl, di.sticky, status, nullptr,
                                        nullptr, KEY_U32, stream);
}

rs_status enqueue_sort(uint32_t* keys, uint32_t* vals, uint32_t n, cudaStream_t stream,
                       void* workspace, size_t workspace_bytes, uint32_t key_type) {
    if (key_type > KEY_F32) return RS_ERR_INVALID_ARG;
    const bool pairs = vals != nullptr;
    const Layout L = layout_for(n, pairs);
    if (workspace == nullptr || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    const ClassKnobs& ck = knobs().cls[size_class(n)];
    // A single small array takes one CTA (one warp alone measured slower);
    // the one-warp sort serves batches of short segments and MSD buckets.
    if (n <= (uint32_t)ck.small_max && n <= small_sort_capacity())
        return launch_small_sort(keys, vals, nullptr, nullptr, nullptr, n, n, ck.small_bits,
                                 key_type, stream);
    // Three passes of 11/11/10-bit digits, where the size class takes them
    // and the caller's workspace holds their buffers.
    if (ck.digits == 11 && key_type == KEY_U32 && workspace_bytes >= layout11(n, pairs).total)
        return enqueue_sort11(keys, vals, n, stream, workspace, workspace_bytes);
    char* ws = static_cast<char*>(workspace);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
    void* status[2] = {ws + L.status0, ws + L.status1};
    const size_t status_bytes = L.status1 - L.status0;
    uint32_t* alt_k = reinterpret_cast<uint32_t*>(ws + L.alt_keys);
    uint32_t* alt_v = pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals) : nullptr;

    // MSD-first order (Alg. 2): tried for unsigned arrays that can split into
    // 256 buckets the one-CTA sort takes; the plan decides on the device
    // from the digit-3 histogram, so the launch sequence stays fixed.
    const bool msd = ck.msd != 0 && key_type == KEY_U32 && n <= kMsdMaxItems;
    uint32_t* msd_off = reinterpret_cast<uint32_t*>(ws + L.msd_off);
    uint32_t* msd_tiny = reinterpret_cast<uint32_t*>(ws + L.msd_tiny);
    uint32_t* msd_small = reinterpret_cast<uint32_t*>(ws + L.msd_small);
    const uint32_t warp_max =
        (uint32_t)ck.warp_max < warp_sort_capacity() ? (uint32_t)ck.warp_max : warp_sort_capacity();

    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return RS_ERR_CUDA;
    st = enqueue_hist4(keys, n, &ctrl->hist[0][0], status[0], status_bytes, key_type, stream);
    if (st != RS_OK) return st;
    note_launch_begin(KK_PLAN, stream);
    const cudaError_t pe = launch_after_previous(k_plan<PASSES>, dim3(1), dim3(1024), 0, stream,
                                                 ctrl, n, msd ? 1u : 0u, warp_max,
                                                 small_sort_capacity(), msd_off, msd_tiny,
                                                 msd_small);
    note_launch_end(KK_PLAN, stream);
    if (pe != cudaSuccess) return RS_ERR_CUDA;

    const int cfg = pairs ? ck.tile_pairs : ck.tile_keys;
    if (msd) {
        // One pass by digit 3 into the alternate buffers (skipped unless the
        // plan chose this order), then every bucket on chip back into the
        // caller's arrays.
        st = pairs ? launch_onesweep_pairs(cfg, false, keys, vals, alt_k, alt_v, n, PASSES - 1,
                                           MSD_SLOT, ctrl, di.sticky, status[0], nullptr, nullptr,
                                           KEY_U32, stream)
                   : launch_onesweep_keys(cfg, false, keys, alt_k, n, PASSES - 1, MSD_SLOT, ctrl,
                                          di.sticky, status[0], nullptr, nullptr, KEY_U32, stream);
        if (st != RS_OK) return st;
        if (warp_max > 0) {
            st = launch_warp_sort(keys, vals, msd_off, msd_tiny, ctrl, 0, ck.small_bits, KEY_U32,
                                  stream, alt_k, alt_v);
            if (st != RS_OK) return st;
        }
        st = launch_small_sort(keys, vals, msd_off, msd_small, ctrl, 0, small_sort_capacity(),
                               ck.small_bits, KEY_U32, stream, alt_k, alt_v);
        if (st != RS_OK) return st;
    }
    for (uint32_t p = 0; p < PASSES; ++p) {
        void* cur = status[p & 1];
        void* next = p + 1 < PASSES ? status[(p + 1) & 1] : nullptr;
        st = pairs ? launch_onesweep_pairs(cfg, L.wide_status, keys, vals, alt_k, alt_v, n, p, p,
                                           ctrl, di.sticky, cur, next, nullptr, key_type, stream)
                   : launch_onesweep_keys(cfg, L.wide_status, keys, alt_k, n, p, p, ctrl, di.sticky,
                                          cur, next, nullptr, key_type, stream);
        if (st != RS_OK) return st;
    }
    return RS_OK;
}

}  // namespace rs
