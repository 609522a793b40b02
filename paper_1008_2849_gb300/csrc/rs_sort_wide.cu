// rs_sort_wide.cu -- sorts of wide items: 64-bit keys (K = 64, D = 8: eight
// passes) carrying no, 32-bit or 64-bit values, and 32-bit keys carrying
// 64-bit values (four passes).  Keys are unsigned or typed (the order-
// preserving maps of rs_device.cuh).  Workspace layout, the histogram and
// plan launches, the scatter passes of 32-bit keys with 64-bit values, and
// the enqueue sequence.
#include "rs_hist_plan.cuh"
#include "rs_internal.h"
#include "rs_onesweep_launch.cuh"

namespace rs {

namespace {

constexpr int HIST8_THREADS = 512;
constexpr int B_WIDE = 2, W_WIDE = 8;

uint32_t wide_tile(bool key64, uint32_t val_bytes) {
    const int items = key64 ? (val_bytes == 8 ? kWideItems64V64 : kWideItems64) : kWideItems32V64;
    return (uint32_t)(kWideThreads * items);
}

template <typename S, bool TYPED>
rs_status pass32v64(uint32_t* ka, unsigned long long* va, uint32_t* kb, unsigned long long* vb,
                    uint32_t n, uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status,
                    void* status_clear, uint32_t key_type, cudaStream_t stream) {
    const SegView none{};
    return launch_onesweep_shape<kWideThreads, kWideItems32V64, B_WIDE, W_WIDE, true, S, false,
                                 TYPED, uint32_t, unsigned long long>(
        ka, va, kb, vb, n, pass, pass, ctrl, sticky, status, status_clear, none, key_type, stream);
}

rs_status launch_pass_k32v64(uint32_t key_type, bool wide, uint32_t* ka, unsigned long long* va,
                             uint32_t* kb, unsigned long long* vb, uint32_t n, uint32_t pass,
                             Ctrl* ctrl, uint32_t* sticky, void* status, void* status_clear,
                             cudaStream_t stream) {
    if (key_type == KEY_U32)
        return wide ? pass32v64<unsigned long long, false>(ka, va, kb, vb, n, pass, ctrl, sticky,
                                                           status, status_clear, KEY_U32, stream)
                    : pass32v64<uint32_t, false>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                                 status_clear, KEY_U32, stream);
    // Typed keys: from typed_split_min items on, the passes that need no
    // maps run without them (see ROLE_PLAIN_PASSES) and both instances are
    // launched for every pass; below it the mapping instance runs them all.
    if (!typed_split(n))
        return wide ? pass32v64<unsigned long long, true>(ka, va, kb, vb, n, pass, ctrl, sticky,
                                                          status, status_clear, key_type, stream)
                    : pass32v64<uint32_t, true>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                                status_clear, key_type, stream);
    const uint32_t plain = key_type | ROLE_PLAIN_PASSES, maps = key_type | ROLE_MAP_PASSES;
    rs_status st = wide ? pass32v64<unsigned long long, false>(ka, va, kb, vb, n, pass, ctrl, sticky,
                                                               status, status_clear, plain, stream)
                        : pass32v64<uint32_t, false>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                                     status_clear, plain, stream);
    if (st != RS_OK) return st;
    return wide ? pass32v64<unsigned long long, true>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                                      status_clear, maps, stream)
                : pass32v64<uint32_t, true>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                            status_clear, maps, stream);
}

}  // namespace

Layout layout_wide(size_t n, bool key64, uint32_t val_bytes) {
    Layout L{};
    const size_t tile = wide_tile(key64, val_bytes);
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
    off = align_up(off + n * (key64 ? 8 : 4), 256);
    L.alt_vals = off;
    off = align_up(off + n * val_bytes, 256);
    L.msd_off = L.msd_tiny = L.msd_small = off;  // no MSD-first order for wide items
    L.total = off;
    return L;
}

rs_status enqueue_sort_wide(void* keys, void* vals, uint32_t n, uint32_t key_type,
                            uint32_t val_bytes, cudaStream_t stream, void* workspace,
                            size_t workspace_bytes) {
    if (key_type > KEY_F64 || (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) ||
        (val_bytes == 0) != (vals == nullptr))
        return RS_ERR_INVALID_ARG;
    const bool key64 = key_type >= KEY_U64;
    if (!key64 && val_bytes != 8) return RS_ERR_INVALID_ARG;  // the 32-bit sorts serve these
    const Layout L = layout_wide(n, key64, val_bytes);
    if (workspace == nullptr || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return RS_ERR_INVALID_ARG;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    char* ws = static_cast<char*>(workspace);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
    void* status[2] = {ws + L.status0, ws + L.status1};
    const size_t status_bytes = L.status1 - L.status0;
    void* alt_k = ws + L.alt_keys;
    void* alt_v = val_bytes ? ws + L.alt_vals : nullptr;
    const uint32_t npass = key64 ? PASSES64 : PASSES;

    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream) != cudaSuccess) return RS_ERR_CUDA;
    if (key64) {
        uint32_t grid = (uint32_t)di.sm_count * 4u;
        const uint32_t need = (n + HIST8_THREADS - 1) / HIST8_THREADS;
        if (grid > need) grid = need;
        auto kern = key_type == KEY_U64 ? k_hist8<HIST8_THREADS, false>
                                        : k_hist8<HIST8_THREADS, true>;
        note_launch_begin(KK_HIST, stream);
        kern<<<grid, HIST8_THREADS, 0, stream>>>(
            static_cast<const unsigned long long*>(keys), n, &ctrl->hist[0][0],
            static_cast<uint4*>(status[0]), (uint32_t)(status_bytes / sizeof(uint4)), key_type);
        note_launch_end(KK_HIST, stream);
        if (cudaPeekAtLastError() != cudaSuccess) return RS_ERR_CUDA;
    } else {
        st = enqueue_hist4(static_cast<const uint32_t*>(keys), n, &ctrl->hist[0][0], status[0],
                           status_bytes, key_type, stream);
        if (st != RS_OK) return st;
    }
    note_launch_begin(KK_PLAN, stream);
    uint32_t* const no_list = nullptr;
    const cudaError_t pe =
        key64 ? launch_after_previous(k_plan<PASSES64>, dim3(1), dim3(1024), 0, stream, ctrl, n,
                                      0u, 0u, 0u, no_list, no_list, no_list)
              : launch_after_previous(k_plan<PASSES>, dim3(1), dim3(1024), 0, stream, ctrl, n, 0u,
                                      0u, 0u, no_list, no_list, no_list);
    note_launch_end(KK_PLAN, stream);
    if (pe != cudaSuccess) return RS_ERR_CUDA;

    for (uint32_t p = 0; p < npass; ++p) {
        void* cur = status[p & 1];
        void* next = p + 1 < npass ? status[(p + 1) & 1] : nullptr;
        if (key64)
            st = launch_pass_k64(key_type, val_bytes, L.wide_status,
                                 static_cast<unsigned long long*>(keys), vals,
                                 static_cast<unsigned long long*>(alt_k), alt_v, n, p, ctrl,
                                 di.sticky, cur, next, stream);
        else
            st = launch_pass_k32v64(key_type, L.wide_status, static_cast<uint32_t*>(keys),
                                    static_cast<unsigned long long*>(vals),
                                    static_cast<uint32_t*>(alt_k),
                                    static_cast<unsigned long long*>(alt_v), n, p, ctrl,
                                    di.sticky, cur, next, stream);
        if (st != RS_OK) return st;
    }
    return RS_OK;
}

}  // namespace rs
