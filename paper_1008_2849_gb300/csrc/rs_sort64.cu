// rs_sort64.cu -- sorts of 64-bit keys (K = 64, D = 8: eight passes),
// optionally carrying 32-bit values: workspace layout, the 64-bit histogram
// and plan launches, and the eight scatter passes.
#include "rs_hist_plan.cuh"
#include "rs_internal.h"
#include "rs_onesweep_launch.cuh"

namespace rs {

namespace {

// Scatter-pass shape of 64-bit keys: 384 threads x 7 keys (a tile of 2688),
// two CTAs per SM, look-back window 8.  The shared-memory plan holds twice
// the key words of a 32-bit tile, hence the shorter tile.
constexpr int T64 = 384, J64 = 7, B64 = 2, W64 = 8;
constexpr uint32_t TILE64 = T64 * J64;
constexpr int HIST8_THREADS = 512;

template <bool PAIRS, typename S>
rs_status launch_pass64(unsigned long long* ka, uint32_t* va, unsigned long long* kb, uint32_t* vb,
                        uint32_t n, uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status,
                        void* status_clear, cudaStream_t stream) {
    const SegView none{};
    return launch_onesweep_shape<T64, J64, B64, W64, PAIRS, S, false, false, unsigned long long>(
        ka, va, kb, vb, n, pass, pass, ctrl, sticky, status, status_clear, none, KEY_U32, stream);
}

}  // namespace

Layout layout_for64(size_t n, bool pairs) {
    Layout L{};
    L.tiles = (uint32_t)((n + TILE64 - 1) / TILE64);
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
    off = align_up(off + n * sizeof(unsigned long long), 256);
    L.alt_vals = off;
    if (pairs) off = align_up(off + n * sizeof(uint32_t), 256);
    L.msd_off = L.msd_tiny = L.msd_small = off;  // no MSD-first order for 64-bit keys
    L.total = off;
    return L;
}

rs_status enqueue_sort64(unsigned long long* keys, uint32_t* vals, uint32_t n, cudaStream_t stream,
                         void* workspace, size_t workspace_bytes) {
    const bool pairs = vals != nullptr;
    const Layout L = layout_for64(n, pairs);
    if (workspace == nullptr || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    char* ws = static_cast<char*>(workspace);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
    void* status[2] = {ws + L.status0, ws + L.status1};
    const size_t status_bytes = L.status1 - L.status0;
    auto* alt_k = reinterpret_cast<unsigned long long*>(ws + L.alt_keys);
    uint32_t* alt_v = pairs ? reinterpret_cast<uint32_t*>(ws + L.alt_vals) : nullptr;

    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return RS_ERR_CUDA;
    uint32_t grid = (uint32_t)di.sm_count * 4u;
    const uint32_t need = (n + HIST8_THREADS - 1) / HIST8_THREADS;
    if (grid > need) grid = need;
    note_launch_begin(KK_HIST, stream);
    k_hist8<HIST8_THREADS><<<grid, HIST8_THREADS, 0, stream>>>(
        keys, n, &ctrl->hist[0][0], static_cast<uint4*>(status[0]),
        (uint32_t)(status_bytes / sizeof(uint4)));
    note_launch_end(KK_HIST, stream);
    note_launch_begin(KK_PLAN, stream);
    k_plan<PASSES64><<<1, 1024, 0, stream>>>(ctrl, n, 0u, 0u, 0u, nullptr, nullptr, nullptr);
    note_launch_end(KK_PLAN, stream);
    if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;

    for (uint32_t p = 0; p < PASSES64; ++p) {
        void* cur = status[p & 1];
        void* next = p + 1 < PASSES64 ? status[(p + 1) & 1] : nullptr;
        if (pairs)
            st = L.wide_status
                     ? launch_pass64<true, unsigned long long>(keys, vals, alt_k, alt_v, n, p, ctrl,
                                                               di.sticky, cur, next, stream)
                     : launch_pass64<true, uint32_t>(keys, vals, alt_k, alt_v, n, p, ctrl,
                                                     di.sticky, cur, next, stream);
        else
            st = L.wide_status
                     ? launch_pass64<false, unsigned long long>(keys, nullptr, alt_k, nullptr, n, p,
                                                                ctrl, di.sticky, cur, next, stream)
                     : launch_pass64<false, uint32_t>(keys, nullptr, alt_k, nullptr, n, p, ctrl,
                                                      di.sticky, cur, next, stream);
        if (st != RS_OK) return st;
    }
    return RS_OK;
}

}  // namespace rs
