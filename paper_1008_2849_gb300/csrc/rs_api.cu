// rs_api.cu -- the extern "C" entry points of librs.so (declared in
// include/rs.h): argument checks, workspace handling for the plain calls,
// the host-buffer path, the sticky device status word, launch counting and
// optional per-kernel event timing.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "rs_device.cuh"
#include "rs_internal.h"

// Sticky status word, one instance per device (a __device__ variable exists
// once in every device's copy of the module).  Host code reaches it only
// through the address cudaGetSymbolAddress returns for the current device.
static __device__ uint32_t g_rs_sticky_err;

namespace rs {

namespace {

constexpr uint32_t kDefaultSpinLimit = 1u << 22;
// Typed sorts below this size launch one scatter-pass instance per pass
// (measured on GB300, float-key pairs as graph replays: one instance is
// 13 % faster at 2^14 items and 5 % at 2^24; two are 1.5 % faster at 2^26).
constexpr uint32_t kDefaultTypedSplitMin = 1u << 25;
constexpr int kMaxDevices = 64;
// Device buffer sets of rs_sort_pairs_host_batch: with three, an array's
// upload never waits for the download of the array two before it.
constexpr int kHostSets = 3;

std::atomic<uint64_t> g_launches{0};

struct DevState {
    bool ready = false;
    DeviceInfo info{};
    // cached workspace of the plain calls
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // cached device buffers and streams of the host-buffer path
    uint32_t* hk = nullptr;
    uint32_t* hv = nullptr;
    size_t h_cap = 0;
    cudaStream_t s_main = nullptr, s_side = nullptr;
    cudaEvent_t ev_vals = nullptr, ev_sorted = nullptr, ev_side_done = nullptr;
    // the pipelined host-buffer path: kHostSets device buffer sets, a
    // copy-in and a copy-out stream (sorts run on s_main), and per set the
    // events that order them
    uint32_t* bk[kHostSets] = {};
    uint32_t* bv[kHostSets] = {};
    size_t b_cap = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kHostSets] = {}, ev_done_sort[kHostSets] = {}, ev_out[kHostSets] = {};
};
DevState g_dev[kMaxDevices];
std::mutex g_mu;       // guards the buffers of g_dev and serialises the plain calls
std::mutex g_info_mu;  // guards g_dev[].ready / .info

// Event timing of launches (benchmark instrumentation).
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_event_pool;
thread_local cudaEvent_t t_pending_begin = nullptr;
thread_local bool t_capturing = false;  // inside rs_graph_create: count, but record no events

cudaEvent_t pool_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return dev;
}

rs_status device_info_for(int dev, DeviceInfo* out) {
    std::lock_guard<std::mutex> lock(g_info_mu);
    DevState& d = g_dev[dev];
    if (!d.ready) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return RS_ERR_CUDA;
        if (major != 10 || minor != 3) return RS_ERR_UNSUPPORTED;  // built for sm_103a only
        void* sticky = nullptr;
        if (cudaGetSymbolAddress(&sticky, g_rs_sticky_err) != cudaSuccess) return RS_ERR_CUDA;
        d.info.sm_count = sms;
        d.info.sticky = static_cast<uint32_t*>(sticky);
        d.ready = true;
    }
    *out = d.info;
    return RS_OK;
}

rs_status ensure_workspace_locked(DevState& d, size_t bytes) {
    if (d.ws_bytes >= bytes) return RS_OK;
    if (d.ws) cudaFree(d.ws);
    d.ws = nullptr;
    d.ws_bytes = 0;
    if (cudaMalloc(&d.ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RS_ERR_OUT_OF_MEMORY;
    }
    d.ws_bytes = bytes;
    return RS_OK;
}

rs_status sticky_status(cudaStream_t stream) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return RS_ERR_CUDA;
    DeviceInfo di;
    rs_status st = device_info(&di);
    if (st != RS_OK) return st;
    uint32_t bits = 0;
    if (cudaMemcpy(&bits, di.sticky, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess)
        return RS_ERR_CUDA;
    if (bits) {
        const uint32_t zero = 0;
        if (cudaMemcpy(di.sticky, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    if (bits & ERR_TIMEOUT) return RS_ERR_TIMEOUT;
    if (bits & ERR_SEGMENTS) return RS_ERR_BAD_SEGMENTS;
    if (bits & ERR_BOUNDS) return RS_ERR_BOUNDS;
    return RS_OK;
}

rs_status plain_sort(uint32_t* keys, uint32_t* vals, size_t n) {
    rs_status st = check_sort_args(keys, vals, n);
    if (st != RS_OK || n == 0) return st;
    std::lock_guard<std::mutex> lock(g_mu);
    const int dev = current_device();
    if (dev < 0) return RS_ERR_CUDA;
    DeviceInfo di;
    st = device_info_for(dev, &di);
    if (st != RS_OK) return st;
    DevState& d = g_dev[dev];
    st = ensure_workspace_locked(d, sort_workspace_bytes(n, vals != nullptr));
    if (st != RS_OK) return st;
    st = enqueue_sort(keys, vals, (uint32_t)n, cudaStreamLegacy, d.ws, d.ws_bytes);
    if (st != RS_OK) return st;
    return sticky_status(cudaStreamLegacy);
}

}  // namespace

size_t sort_workspace_bytes(size_t n, bool pairs) {
    size_t t = layout_for(n, pairs).total;
    if (n > 0 && n < (size_t(1) << 32) && knobs().cls[size_class(n)].digits == 11) {
        const size_t t11 = layout11(n, pairs).total;
        if (t11 > t) t = t11;
    }
    return t;
}

rs_status check_sort_args(const uint32_t* keys, const uint32_t* vals, size_t n) {
    if (n >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
    if (n > 0 && keys == nullptr) return RS_ERR_INVALID_ARG;
    if (vals != nullptr && n > 0) {
        const uintptr_t k0 = (uintptr_t)keys, k1 = k0 + n * 4;
        const uintptr_t v0 = (uintptr_t)vals, v1 = v0 + n * 4;
        if (k0 < v1 && v0 < k1) return RS_ERR_INVALID_ARG;  // overlapping
    }
    if (((uintptr_t)keys & 3u) || ((uintptr_t)vals & 3u)) return RS_ERR_INVALID_ARG;
    return RS_OK;
}

Knobs& knobs() {
    // Defaults chosen by the autotuner on GB300 (tuning_gb300.json): arrays up
    // to 8192 items take the one-CTA sort; up to 2^20 items tile shape 1
    // (512 x 8, two CTAs per SM); larger ones shape 3 (384 x 13, two CTAs per
    // SM), and for keys only shape 6 (384 x 18: no value buffer, still two
    // CTAs).
    // Per class:
    // {tile_pairs, tile_keys, tile_seg, small_max, warp_max, small_bits, msd,
    //  digits}.
    // The MSD-first order measured faster only up to 2^16 items (class 1).
    // The 11-bit-digit order (three passes) measured slower in every class
    // (2.3 to 2.8 times the 8-bit sort at 2^24 to 2^28 pairs), so it is off.
    static Knobs k{{{1, 1, 3, 8192, 512, 8, 0, 8}, {1, 1, 3, 4096, 512, 8, 1, 8},
                    {1, 1, 3, 4096, 512, 8, 0, 8}, {3, 6, 3, 4096, 512, 8, 0, 8},
                    {3, 6, 3, 4096, 512, 8, 0, 8}, {3, 6, 3, 4096, 512, 8, 0, 8}},
                   kDefaultSpinLimit, 0, 4, 3, kDefaultTypedSplitMin, 1, 1};
    return k;
}

int size_class(size_t items) {
    if (items <= (size_t(1) << 13)) return 0;
    if (items <= (size_t(1) << 16)) return 1;
    if (items <= (size_t(1) << 20)) return 2;
    if (items <= (size_t(1) << 24)) return 3;
    if (items <= (size_t(1) << 28)) return 4;
    return 5;
}

const char* kernel_kind_name(int kind) {
    switch (kind) {
    case KK_HIST: return "hist4";
    case KK_PLAN: return "plan";
    case KK_ONESWEEP: return "onesweep";
    case KK_SMALL: return "small_sort";
    case KK_SEG_PLAN: return "seg_plan";
    case KK_SEG_HIST: return "seg_hist";
    case KK_SEG_SCAN: return "seg_scan";
    case KK_SEG_ONESWEEP: return "seg_onesweep";
    case KK_WARP: return "warp_sort";
    case KK_D11_UP: return "d11_up";
    case KK_D11_SCAN: return "d11_scan";
    case KK_D11_DOWN: return "d11_down";
    default: return nullptr;
    }
}

rs_status device_info(DeviceInfo* out) {
    const int dev = current_device();
    if (dev < 0) return RS_ERR_CUDA;
    return device_info_for(dev, out);
}

void note_launch_begin(int kind, cudaStream_t stream) {
    (void)kind;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on || t_capturing) return;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (!g_prof_on) return;
    t_pending_begin = pool_event();
    cudaEventRecord(t_pending_begin, stream);
}

void note_launch_end(int kind, cudaStream_t stream) {
    if (t_pending_begin == nullptr) return;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    cudaEvent_t b = pool_event();
    cudaEventRecord(b, stream);
    g_prof_recs.push_back(ProfRec{kind, t_pending_begin, b});
    t_pending_begin = nullptr;
}

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_sort_keys(uint32_t* d_keys, size_t n) { return plain_sort(d_keys, nullptr, n); }

rs_status rs_sort_pairs(uint32_t* d_keys, uint32_t* d_vals, size_t n) {
    if (n > 0 && d_vals == nullptr) return RS_ERR_INVALID_ARG;
    return plain_sort(d_keys, d_vals, n);
}

static rs_status ex_sort(uint32_t* keys, uint32_t* vals, size_t n, void* stream, void* ws,
                         size_t ws_bytes, int key_type = RS_KEY_U32) {
    if (key_type < RS_KEY_U32 || key_type > RS_KEY_F32) return RS_ERR_INVALID_ARG;
    rs_status st = check_sort_args(keys, vals, n);
    if (st != RS_OK || n == 0) return st;
    if (ws_bytes < layout_for(n, vals != nullptr).total || ws == nullptr) return RS_ERR_INVALID_ARG;
    return enqueue_sort(keys, vals, (uint32_t)n, static_cast<cudaStream_t>(stream), ws, ws_bytes,
                        (uint32_t)key_type);
}

rs_status rs_sort_keys_ex(uint32_t* d_keys, size_t n, void* cuda_stream, void* d_workspace,
                          size_t workspace_bytes) {
    return ex_sort(d_keys, nullptr, n, cuda_stream, d_workspace, workspace_bytes);
}

rs_status rs_sort_pairs_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n, void* cuda_stream,
                           void* d_workspace, size_t workspace_bytes) {
    if (n > 0 && d_vals == nullptr) return RS_ERR_INVALID_ARG;
    return ex_sort(d_keys, d_vals, n, cuda_stream, d_workspace, workspace_bytes);
}

size_t rs_workspace_bytes_digits11(size_t n, int with_values) {
    if (n == 0 || n >= (size_t(1) << 32)) return 0;
    return layout11(n, with_values != 0).total;
}

rs_status rs_sort_digits11_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n, void* cuda_stream,
                              void* d_workspace, size_t workspace_bytes) {
    rs_status st = check_sort_args(d_keys, d_vals, n);
    if (st != RS_OK || n == 0) return st;
    if (d_workspace == nullptr || workspace_bytes < layout11(n, d_vals != nullptr).total)
        return RS_ERR_INVALID_ARG;
    return enqueue_sort11(d_keys, d_vals, (uint32_t)n, static_cast<cudaStream_t>(cuda_stream),
                          d_workspace, workspace_bytes);
}

static rs_status seg_args(const uint32_t* keys, const uint32_t* vals, size_t n,
                          const uint32_t* offsets, uint32_t num_segments) {
    rs_status st = check_sort_args(keys, vals, n);
    if (st != RS_OK) return st;
    if (num_segments > 0 && offsets == nullptr) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)offsets & 3u)) return RS_ERR_INVALID_ARG;
    return RS_OK;
}

static rs_status plain_segmented(uint32_t* keys, uint32_t* vals, size_t n,
                                 const uint32_t* offsets, uint32_t num_segments) {
    rs_status st = seg_args(keys, vals, n, offsets, num_segments);
    if (st != RS_OK || n == 0 || num_segments == 0) return st;
    std::lock_guard<std::mutex> lock(g_mu);
    const int dev = current_device();
    if (dev < 0) return RS_ERR_CUDA;
    DeviceInfo di;
    st = device_info_for(dev, &di);
    if (st != RS_OK) return st;
    DevState& d = g_dev[dev];
    st = ensure_workspace_locked(d, seg_layout_for(n, vals != nullptr, num_segments).total);
    if (st != RS_OK) return st;
    st = enqueue_sort_segmented(keys, vals, (uint32_t)n, offsets, num_segments, cudaStreamLegacy,
                                d.ws, d.ws_bytes);
    if (st != RS_OK) return st;
    return sticky_status(cudaStreamLegacy);
}

rs_status rs_sort_keys_segmented(uint32_t* d_keys, size_t n, const uint32_t* d_offsets,
                                 uint32_t num_segments) {
    return plain_segmented(d_keys, nullptr, n, d_offsets, num_segments);
}

rs_status rs_sort_pairs_segmented(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                  const uint32_t* d_offsets, uint32_t num_segments) {
    if (n > 0 && d_vals == nullptr) return RS_ERR_INVALID_ARG;
    return plain_segmented(d_keys, d_vals, n, d_offsets, num_segments);
}

static rs_status ex_segmented(uint32_t* keys, uint32_t* vals, size_t n, const uint32_t* offsets,
                              uint32_t num_segments, void* stream, void* ws, size_t ws_bytes,
                              int key_type = RS_KEY_U32) {
    if (key_type < RS_KEY_U32 || key_type > RS_KEY_F32) return RS_ERR_INVALID_ARG;
    rs_status st = seg_args(keys, vals, n, offsets, num_segments);
    if (st != RS_OK || n == 0 || num_segments == 0) return st;
    if (ws == nullptr || ws_bytes < seg_layout_for(n, vals != nullptr, num_segments).total)
        return RS_ERR_INVALID_ARG;
    return enqueue_sort_segmented(keys, vals, (uint32_t)n, offsets, num_segments,
                                  static_cast<cudaStream_t>(stream), ws, ws_bytes,
                                  (uint32_t)key_type);
}

rs_status rs_sort_typed_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n, int key_type,
                           void* cuda_stream, void* d_workspace, size_t workspace_bytes) {
    return ex_sort(d_keys, d_vals, n, cuda_stream, d_workspace, workspace_bytes, key_type);
}

rs_status rs_sort_segmented_typed_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                     const uint32_t* d_offsets, uint32_t num_segments,
                                     int key_type, void* cuda_stream, void* d_workspace,
                                     size_t workspace_bytes) {
    return ex_segmented(d_keys, d_vals, n, d_offsets, num_segments, cuda_stream, d_workspace,
                        workspace_bytes, key_type);
}

rs_status rs_sort_keys_segmented_ex(uint32_t* d_keys, size_t n, const uint32_t* d_offsets,
                                    uint32_t num_segments, void* cuda_stream, void* d_workspace,
                                    size_t workspace_bytes) {
    return ex_segmented(d_keys, nullptr, n, d_offsets, num_segments, cuda_stream, d_workspace,
                        workspace_bytes);
}

rs_status rs_sort_pairs_segmented_ex(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                     const uint32_t* d_offsets, uint32_t num_segments,
                                     void* cuda_stream, void* d_workspace,
                                     size_t workspace_bytes) {
    if (n > 0 && d_vals == nullptr) return RS_ERR_INVALID_ARG;
    return ex_segmented(d_keys, d_vals, n, d_offsets, num_segments, cuda_stream, d_workspace,
                        workspace_bytes);
}

size_t rs_workspace_bytes(size_t n, int with_values, uint32_t num_segments) {
    if (n == 0) return 0;
    if (num_segments > 0) return seg_layout_for(n, with_values != 0, num_segments).total;
    return sort_workspace_bytes(n, with_values != 0);
}

size_t rs_workspace_bytes64(size_t n, int with_values) {
    if (n == 0) return 0;
    return layout_wide(n, true, with_values ? 4u : 0u).total;
}

rs_status rs_sort64_ex(uint64_t* d_keys, uint32_t* d_vals, size_t n, void* cuda_stream,
                       void* d_workspace, size_t workspace_bytes) {
    return rs_sort_kv_ex(d_keys, d_vals, n, RS_KEY_U64, d_vals != nullptr ? 32 : 0, cuda_stream,
                         d_workspace, workspace_bytes);
}

namespace {

bool valid_kv_types(int key_type, int value_bits) {
    return key_type >= RS_KEY_U32 && key_type <= RS_KEY_F64 &&
           (value_bits == 0 || value_bits == 32 || value_bits == 64);
}

// The 32-bit sorts (autotuned shapes, on-chip sorts of small arrays) serve
// 32-bit keys with no or 32-bit values; everything else is a wide sort.
bool kv_is_narrow(int key_type, int value_bits) {
    return key_type <= RS_KEY_F32 && value_bits <= 32;
}

}  // namespace

size_t rs_workspace_bytes_kv(size_t n, int key_type, int value_bits) {
    if (n == 0 || !valid_kv_types(key_type, value_bits)) return 0;
    if (kv_is_narrow(key_type, value_bits)) return layout_for(n, value_bits != 0).total;
    return layout_wide(n, key_type >= RS_KEY_U64, (uint32_t)value_bits / 8).total;
}

rs_status rs_sort_kv_ex(void* d_keys, void* d_vals, size_t n, int key_type, int value_bits,
                        void* cuda_stream, void* d_workspace, size_t workspace_bytes) {
    if (!valid_kv_types(key_type, value_bits)) return RS_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
    if (n == 0) return RS_OK;
    if (kv_is_narrow(key_type, value_bits)) {
        if ((value_bits == 0) != (d_vals == nullptr)) return RS_ERR_INVALID_ARG;
        return ex_sort(static_cast<uint32_t*>(d_keys), static_cast<uint32_t*>(d_vals), n,
                       cuda_stream, d_workspace, workspace_bytes, key_type);
    }
    const size_t kb = key_type >= RS_KEY_U64 ? 8 : 4, vb = (size_t)value_bits / 8;
    if (d_keys == nullptr || (vb == 0) != (d_vals == nullptr)) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)d_keys & (kb - 1)) || (vb && ((uintptr_t)d_vals & (vb - 1))))
        return RS_ERR_INVALID_ARG;
    if (vb) {
        const uintptr_t k0 = (uintptr_t)d_keys, k1 = k0 + n * kb;
        const uintptr_t v0 = (uintptr_t)d_vals, v1 = v0 + n * vb;
        if (k0 < v1 && v0 < k1) return RS_ERR_INVALID_ARG;  // overlapping
    }
    if (d_workspace == nullptr ||
        workspace_bytes < layout_wide(n, kb == 8, (uint32_t)vb).total)
        return RS_ERR_INVALID_ARG;
    return enqueue_sort_wide(d_keys, d_vals, (uint32_t)n, (uint32_t)key_type, (uint32_t)vb,
                             static_cast<cudaStream_t>(cuda_stream), d_workspace,
                             workspace_bytes);
}

size_t rs_workspace_bytes_kv_segmented(size_t n, int key_type, int value_bits,
                                       uint32_t num_segments) {
    if (n == 0 || num_segments == 0 || !valid_kv_types(key_type, value_bits)) return 0;
    if (kv_is_narrow(key_type, value_bits))
        return seg_layout_for(n, value_bits != 0, num_segments).total;
    return seg_layout_wide(n, key_type >= RS_KEY_U64, (uint32_t)value_bits / 8, num_segments)
        .total;
}

rs_status rs_sort_kv_segmented_ex(void* d_keys, void* d_vals, size_t n, const uint32_t* d_offsets,
                                  uint32_t num_segments, int key_type, int value_bits,
                                  void* cuda_stream, void* d_workspace, size_t workspace_bytes) {
    if (!valid_kv_types(key_type, value_bits)) return RS_ERR_INVALID_ARG;
    if (n >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
    if (kv_is_narrow(key_type, value_bits)) {
        if ((value_bits == 0) != (d_vals == nullptr)) return RS_ERR_INVALID_ARG;
        return ex_segmented(static_cast<uint32_t*>(d_keys), static_cast<uint32_t*>(d_vals), n,
                            d_offsets, num_segments, cuda_stream, d_workspace, workspace_bytes,
                            key_type);
    }
    const size_t kb = key_type >= RS_KEY_U64 ? 8 : 4, vb = (size_t)value_bits / 8;
    if ((vb == 0) != (d_vals == nullptr)) return RS_ERR_INVALID_ARG;
    if (n == 0 || num_segments == 0) return RS_OK;
    if (d_keys == nullptr || d_offsets == nullptr || ((uintptr_t)d_offsets & 3u))
        return RS_ERR_INVALID_ARG;
    if (((uintptr_t)d_keys & (kb - 1)) || (vb && ((uintptr_t)d_vals & (vb - 1))))
        return RS_ERR_INVALID_ARG;
    if (vb) {
        const uintptr_t k0 = (uintptr_t)d_keys, k1 = k0 + n * kb;
        const uintptr_t v0 = (uintptr_t)d_vals, v1 = v0 + n * vb;
        if (k0 < v1 && v0 < k1) return RS_ERR_INVALID_ARG;  // overlapping
    }
    if (d_workspace == nullptr ||
        workspace_bytes < seg_layout_wide(n, kb == 8, (uint32_t)vb, num_segments).total)
        return RS_ERR_INVALID_ARG;
    return enqueue_sort_segmented_wide(d_keys, d_vals, (uint32_t)n, d_offsets, num_segments,
                                       (uint32_t)key_type, (uint32_t)vb,
                                       static_cast<cudaStream_t>(cuda_stream), d_workspace,
                                       workspace_bytes);
}

rs_status rs_stream_status(void* cuda_stream) {
    return sticky_status(static_cast<cudaStream_t>(cuda_stream));
}

const char* rs_status_string(rs_status status) {
    switch (status) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_OUT_OF_MEMORY: return "out of device memory";
    case RS_ERR_CUDA: return "CUDA runtime error";
    case RS_ERR_TIMEOUT: return "device-side wait timed out";
    case RS_ERR_UNSUPPORTED: return "unsupported device or size";
    case RS_ERR_BOUNDS: return "device-side bounds check refused a write";
    case RS_ERR_BAD_SEGMENTS: return "malformed segment table";
    default: return "unknown status";
    }
}

rs_status rs_msd_partition_ex(const uint32_t* d_keys, const uint32_t* d_vals, size_t n,
                               uint32_t* d_out_keys, uint32_t* d_out_vals,
                               uint32_t* d_bucket_offsets, void* cuda_stream, void* d_workspace,
                               size_t workspace_bytes) {
    if (n >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
    if (d_bucket_offsets == nullptr || ((uintptr_t)d_bucket_offsets & 3u))
        return RS_ERR_INVALID_ARG;
    if ((d_vals == nullptr) != (d_out_vals == nullptr)) return RS_ERR_INVALID_ARG;
    rs_status st = check_sort_args(d_keys, d_vals, n);
    if (st != RS_OK) return st;
    st = check_sort_args(d_out_keys, d_out_vals, n);
    if (st != RS_OK) return st;
    if (n > 0) {  // outputs apart from the inputs
        auto apart = [n](const void* a, const void* b) {
            const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b, len = n * sizeof(uint32_t);
            return a == nullptr || b == nullptr || x + len <= y || y + len <= x;
        };
        if (!apart(d_keys, d_out_keys) || !apart(d_keys, d_out_vals) ||
            !apart(d_vals, d_out_keys) || !apart(d_vals, d_out_vals))
            return RS_ERR_INVALID_ARG;
    }
    const cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (n == 0) {
        return cudaMemsetAsync(d_bucket_offsets, 0, 257 * sizeof(uint32_t), stream) ==
                       cudaSuccess
                   ? RS_OK
                   : RS_ERR_CUDA;
    }
    if (d_workspace == nullptr || workspace_bytes < layout_for(n, d_vals != nullptr).total)
        return RS_ERR_INVALID_ARG;
    return enqueue_msd_partition(d_keys, d_vals, (uint32_t)n, d_out_keys, d_out_vals,
                                 d_bucket_offsets, stream, d_workspace, workspace_bytes);
}

rs_status rs_digit_histograms_ex(const uint32_t* d_keys, size_t n, uint32_t* d_hist,
                                 void* cuda_stream) {
    if (n >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
    if (d_hist == nullptr || (n > 0 && d_keys == nullptr)) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)d_keys & 3u) || ((uintptr_t)d_hist & 3u)) return RS_ERR_INVALID_ARG;
    return enqueue_histograms(d_keys, (uint32_t)n, d_hist, static_cast<cudaStream_t>(cuda_stream));
}

rs_status rs_sort_pairs_host(const uint32_t* h_keys_in, const uint32_t* h_vals_in,
                             uint32_t* h_keys_out, uint32_t* h_vals_out, size_t n) {
    if (n >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
    if (n == 0) return RS_OK;
    if (!h_keys_in || !h_keys_out || (h_vals_in && !h_vals_out)) return RS_ERR_INVALID_ARG;
    const bool pairs = h_vals_in != nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    const int dev = current_device();
    if (dev < 0) return RS_ERR_CUDA;
    DeviceInfo di;
    rs_status st = device_info_for(dev, &di);
    if (st != RS_OK) return st;
    DevState& d = g_dev[dev];
    if (!d.s_main) {
        if (cudaStreamCreateWithFlags(&d.s_main, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&d.s_side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&d.ev_vals, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&d.ev_sorted, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&d.ev_side_done, cudaEventDisableTiming) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    if (d.h_cap < n) {
        if (d.hk) cudaFree(d.hk);
        if (d.hv) cudaFree(d.hv);
        d.hk = d.hv = nullptr;
        d.h_cap = 0;
        if (cudaMalloc(&d.hk, n * 4) != cudaSuccess || cudaMalloc(&d.hv, n * 4) != cudaSuccess) {
            cudaGetLastError();
            return RS_ERR_OUT_OF_MEMORY;
        }
        d.h_cap = n;
    }
    st = ensure_workspace_locked(d, sort_workspace_bytes(n, pairs));
    if (st != RS_OK) return st;
    const size_t bytes = n * 4;
    // A failure part-way waits for the work already enqueued, so that no copy
    // still reads or writes the caller's arrays.
    auto drain = [&](rs_status e) {
        cudaStreamSynchronize(d.s_side);
        cudaStreamSynchronize(d.s_main);
        return e;
    };
    // Keys first on the main stream (the histogram needs them); values on
    // the side stream, overlapping the histogram and plan kernels.
    if (cudaMemcpyAsync(d.hk, h_keys_in, bytes, cudaMemcpyHostToDevice, d.s_main) != cudaSuccess)
        return drain(RS_ERR_CUDA);
    if (pairs) {
        if (cudaMemcpyAsync(d.hv, h_vals_in, bytes, cudaMemcpyHostToDevice, d.s_side) != cudaSuccess ||
            cudaEventRecord(d.ev_vals, d.s_side) != cudaSuccess ||
            cudaStreamWaitEvent(d.s_main, d.ev_vals, 0) != cudaSuccess)
            return drain(RS_ERR_CUDA);
    }
    st = enqueue_sort(d.hk, pairs ? d.hv : nullptr, (uint32_t)n, d.s_main, d.ws, d.ws_bytes);
    if (st != RS_OK) return drain(st);
    if (pairs) {
        if (cudaEventRecord(d.ev_sorted, d.s_main) != cudaSuccess ||
            cudaStreamWaitEvent(d.s_side, d.ev_sorted, 0) != cudaSuccess ||
            cudaMemcpyAsync(h_vals_out, d.hv, bytes, cudaMemcpyDeviceToHost, d.s_side) != cudaSuccess)
            return drain(RS_ERR_CUDA);
    }
    if (cudaMemcpyAsync(h_keys_out, d.hk, bytes, cudaMemcpyDeviceToHost, d.s_main) != cudaSuccess)
        return drain(RS_ERR_CUDA);
    if (cudaStreamSynchronize(d.s_side) != cudaSuccess) return drain(RS_ERR_CUDA);
    return sticky_status(d.s_main);
}

rs_status rs_sort_pairs_host_batch(const uint32_t* const* h_keys_in,
                                   const uint32_t* const* h_vals_in, uint32_t* const* h_keys_out,
                                   uint32_t* const* h_vals_out, const size_t* n, uint32_t count) {
    if (count == 0) return RS_OK;
    if (!h_keys_in || !h_keys_out || !n || (h_vals_in && !h_vals_out)) return RS_ERR_INVALID_ARG;
    const bool pairs = h_vals_in != nullptr;
    size_t nmax = 0;
    for (uint32_t i = 0; i < count; ++i) {
        if (n[i] >= (size_t(1) << 32)) return RS_ERR_UNSUPPORTED;
        if (n[i] == 0) continue;
        if (!h_keys_in[i] || !h_keys_out[i] || (pairs && (!h_vals_in[i] || !h_vals_out[i])))
            return RS_ERR_INVALID_ARG;
        if (n[i] > nmax) nmax = n[i];
    }
    if (nmax == 0) return RS_OK;
    std::lock_guard<std::mutex> lock(g_mu);
    const int dev = current_device();
    if (dev < 0) return RS_ERR_CUDA;
    DeviceInfo di;
    rs_status st = device_info_for(dev, &di);
    if (st != RS_OK) return st;
    DevState& d = g_dev[dev];
    if (!d.s_main) {
        if (cudaStreamCreateWithFlags(&d.s_main, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&d.s_side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&d.ev_vals, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&d.ev_sorted, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&d.ev_side_done, cudaEventDisableTiming) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    if (!d.s_in) {
        if (cudaStreamCreateWithFlags(&d.s_in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&d.s_out, cudaStreamNonBlocking) != cudaSuccess)
            return RS_ERR_CUDA;
        for (int b = 0; b < kHostSets; ++b)
            if (cudaEventCreateWithFlags(&d.ev_in[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&d.ev_done_sort[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&d.ev_out[b], cudaEventDisableTiming) != cudaSuccess)
                return RS_ERR_CUDA;
    }
    if (d.b_cap < nmax) {
        for (int b = 0; b < kHostSets; ++b) {
            if (d.bk[b]) cudaFree(d.bk[b]);
            if (d.bv[b]) cudaFree(d.bv[b]);
            d.bk[b] = d.bv[b] = nullptr;
        }
        d.b_cap = 0;
        for (int b = 0; b < kHostSets; ++b)
            if (cudaMalloc(&d.bk[b], nmax * 4) != cudaSuccess ||
                cudaMalloc(&d.bv[b], nmax * 4) != cudaSuccess) {
                cudaGetLastError();
                return RS_ERR_OUT_OF_MEMORY;
            }
        d.b_cap = nmax;
    }
    size_t ws_need = 0;
    for (uint32_t i = 0; i < count; ++i)
        if (n[i] > 0) ws_need = std::max(ws_need, sort_workspace_bytes(n[i], pairs));
    st = ensure_workspace_locked(d, ws_need);
    if (st != RS_OK) return st;
    // Array i uses buffer set i % kHostSets.  Its upload waits for the
    // download of the array that used the set before; its sort (one compute
    // stream, one workspace) waits for its upload; its download waits for its
    // sort.  So the next array's upload and the previous one's download run
    // while array i is sorted.  A failure part-way waits for the work already
    // enqueued, so that no copy still reads or writes the caller's arrays.
    auto drain = [&](rs_status e) {
        cudaStreamSynchronize(d.s_in);
        cudaStreamSynchronize(d.s_main);
        cudaStreamSynchronize(d.s_out);
        return e;
    };
    for (uint32_t i = 0; i < count; ++i) {
        if (n[i] == 0) continue;
        const int b = (int)(i % kHostSets);
        const size_t bytes = n[i] * 4;
        if (cudaStreamWaitEvent(d.s_in, d.ev_out[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(d.bk[b], h_keys_in[i], bytes, cudaMemcpyHostToDevice, d.s_in) !=
                cudaSuccess ||
            (pairs && cudaMemcpyAsync(d.bv[b], h_vals_in[i], bytes, cudaMemcpyHostToDevice,
                                      d.s_in) != cudaSuccess) ||
            cudaEventRecord(d.ev_in[b], d.s_in) != cudaSuccess ||
            cudaStreamWaitEvent(d.s_main, d.ev_in[b], 0) != cudaSuccess)
            return drain(RS_ERR_CUDA);
        st = enqueue_sort(d.bk[b], pairs ? d.bv[b] : nullptr, (uint32_t)n[i], d.s_main, d.ws,
                          d.ws_bytes);
        if (st != RS_OK) return drain(st);
        if (cudaEventRecord(d.ev_done_sort[b], d.s_main) != cudaSuccess ||
            cudaStreamWaitEvent(d.s_out, d.ev_done_sort[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(h_keys_out[i], d.bk[b], bytes, cudaMemcpyDeviceToHost, d.s_out) !=
                cudaSuccess ||
            (pairs && cudaMemcpyAsync(h_vals_out[i], d.bv[b], bytes, cudaMemcpyDeviceToHost,
                                      d.s_out) != cudaSuccess) ||
            cudaEventRecord(d.ev_out[b], d.s_out) != cudaSuccess)
            return drain(RS_ERR_CUDA);
    }
    if (cudaStreamSynchronize(d.s_out) != cudaSuccess || cudaStreamSynchronize(d.s_in) != cudaSuccess)
        return drain(RS_ERR_CUDA);
    return sticky_status(d.s_main);
}

}  // extern "C"

struct rs_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;  // kernels per replay (for rs_launch_count)
};

extern "C" {

rs_status rs_graph_create(rs_graph* out, uint32_t* d_keys, uint32_t* d_vals, size_t n,
                          const uint32_t* d_offsets, uint32_t num_segments, void* d_workspace,
                          size_t workspace_bytes) {
    if (out == nullptr || n == 0) return RS_ERR_INVALID_ARG;
    *out = nullptr;
    rs_status st = num_segments ? seg_args(d_keys, d_vals, n, d_offsets, num_segments)
                                : check_sort_args(d_keys, d_vals, n);
    if (st != RS_OK) return st;
    const size_t need = num_segments ? seg_layout_for(n, d_vals != nullptr, num_segments).total
                                     : layout_for(n, d_vals != nullptr).total;
    if (d_workspace == nullptr || workspace_bytes < need) return RS_ERR_INVALID_ARG;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RS_ERR_CUDA;
    rs_graph_s* g = new rs_graph_s();
    const uint64_t before = g_launches.load(std::memory_order_relaxed);
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(s);
        delete g;
        return RS_ERR_CUDA;
    }
    t_capturing = true;
    st = num_segments ? enqueue_sort_segmented(d_keys, d_vals, (uint32_t)n, d_offsets, num_segments,
                                               s, d_workspace, workspace_bytes)
                      : enqueue_sort(d_keys, d_vals, (uint32_t)n, s, d_workspace, workspace_bytes);
    t_capturing = false;
    const cudaError_t ce = cudaStreamEndCapture(s, &g->graph);
    g->kernels = g_launches.load(std::memory_order_relaxed) - before;
    g_launches.fetch_sub(g->kernels, std::memory_order_relaxed);  // captured, not launched
    cudaStreamDestroy(s);
    if (st == RS_OK && ce != cudaSuccess) st = RS_ERR_CUDA;
    if (st == RS_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) st = RS_ERR_CUDA;
    if (st != RS_OK) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        cudaGetLastError();
        return st;
    }
    *out = g;
    return RS_OK;
}

rs_status rs_graph_launch(rs_graph graph, void* cuda_stream) {
    if (graph == nullptr) return RS_ERR_INVALID_ARG;
    if (cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
        return RS_ERR_CUDA;
    g_launches.fetch_add(graph->kernels, std::memory_order_relaxed);
    return RS_OK;
}

rs_status rs_graph_destroy(rs_graph graph) {
    if (graph == nullptr) return RS_ERR_INVALID_ARG;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return RS_OK;
}

uint64_t rs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

rs_status rs_profile_enable(int on) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_on = on != 0;
    if (!g_prof_on) {
        for (auto& r : g_prof_recs) {
            g_event_pool.push_back(r.a);
            g_event_pool.push_back(r.b);
        }
        g_prof_recs.clear();
    }
    return RS_OK;
}

int rs_profile_read(uint64_t* launches, double* total_ms, int max_kinds) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    for (int k = 0; k < max_kinds && k < KK_COUNT; ++k) {
        if (launches) launches[k] = 0;
        if (total_ms) total_ms[k] = 0.0;
    }
    for (auto& r : g_prof_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        if (r.kind < max_kinds) {
            if (launches) launches[r.kind] += 1;
            if (total_ms) total_ms[r.kind] += ms;
        }
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_prof_recs.clear();
    return KK_COUNT;
}

const char* rs_kernel_kind_name(int kind) { return kernel_kind_name(kind); }

static rs_status set_class_knob(ClassKnobs& c, int knob, int value) {
    switch (knob) {
    case 0:
    case 1:
    case 5:
        if (value < 0 || value >= NUM_TILE_CONFIGS) return RS_ERR_INVALID_ARG;
        (knob == 0 ? c.tile_pairs : knob == 1 ? c.tile_keys : c.tile_seg) = value;
        return RS_OK;
    case 4:
        if (value < 0 || value > (int)small_sort_capacity()) return RS_ERR_INVALID_ARG;
        c.small_max = value;
        return RS_OK;
    case 6:
        if (value < 0 || value > (int)warp_sort_capacity()) return RS_ERR_INVALID_ARG;
        c.warp_max = value;
        return RS_OK;
    case 7:
        if (value != 4 && value != 8) return RS_ERR_INVALID_ARG;
        c.small_bits = value;
        return RS_OK;
    case 8:
        if (value != 0 && value != 1) return RS_ERR_INVALID_ARG;
        c.msd = value;
        return RS_OK;
    case 11:
        if (value != 8 && value != 11) return RS_ERR_INVALID_ARG;
        c.digits = value;
        return RS_OK;
    default: return RS_ERR_INVALID_ARG;
    }
}

static int get_class_knob(const ClassKnobs& c, int knob) {
    switch (knob) {
    case 0: return c.tile_pairs;
    case 1: return c.tile_keys;
    case 4: return c.small_max;
    case 5: return c.tile_seg;
    case 6: return c.warp_max;
    case 7: return c.small_bits;
    case 8: return c.msd;
    case 11: return c.digits;
    default: return -1;
    }
}

rs_status rs_tune_set(int knob, int value) {
    Knobs& k = knobs();
    switch (knob) {
    case 2:
        if (value < 1 || value > 16) return RS_ERR_INVALID_ARG;
        k.hist_ctas_per_sm = value;
        return RS_OK;
    case 3:
        if (value < 0 || value > 3) return RS_ERR_INVALID_ARG;
        k.hist_mode = value;
        return RS_OK;
    case 9:
        if (value < 0) return RS_ERR_INVALID_ARG;
        k.typed_split_min = (uint32_t)value;
        return RS_OK;
    case 10:
        if (value < 0 || value >= d11_shape_count()) return RS_ERR_INVALID_ARG;
        k.d11_shape = value;
        return RS_OK;
    case 13:
        if (value != 0 && value != 1) return RS_ERR_INVALID_ARG;
        k.pdl = value;
        return RS_OK;
    default:
        for (int c = 0; c < NUM_SIZE_CLASSES; ++c) {
            rs_status st = set_class_knob(k.cls[c], knob, value);
            if (st != RS_OK) return st;
        }
        return RS_OK;
    }
}

int rs_tune_get(int knob) {
    const Knobs& k = knobs();
    switch (knob) {
    case 2: return k.hist_ctas_per_sm;
    case 3: return k.hist_mode;
    case 9: return (int)(k.typed_split_min > 0x7fffffffu ? 0x7fffffffu : k.typed_split_min);
    case 10: return k.d11_shape;
    case 13: return k.pdl;
    default: return get_class_knob(k.cls[4], knob);
    }
}

rs_status rs_tune_set_class(int size_class_index, int knob, int value) {
    if (size_class_index < 0 || size_class_index >= NUM_SIZE_CLASSES) return RS_ERR_INVALID_ARG;
    return set_class_knob(knobs().cls[size_class_index], knob, value);
}

int rs_tune_get_class(int size_class_index, int knob) {
    if (size_class_index < 0 || size_class_index >= NUM_SIZE_CLASSES) return -1;
    return get_class_knob(knobs().cls[size_class_index], knob);
}

int rs_size_class(size_t items) { return size_class(items); }

int rs_tile_shape_count(void) { return NUM_TILE_CONFIGS; }

rs_status rs_tile_shape(int index, int* threads, int* items_per_thread) {
    if (index < 0 || index >= NUM_TILE_CONFIGS) return RS_ERR_INVALID_ARG;
    if (threads) *threads = kTileConfigs[index].threads;
    if (items_per_thread) *items_per_thread = kTileConfigs[index].items;
    return RS_OK;
}

rs_status rs_debug_set_spin_limit(uint32_t iterations) {
    knobs().spin_limit = iterations ? iterations : kDefaultSpinLimit;
    return RS_OK;
}

rs_status rs_debug_withhold_first_tile(int withhold) {
    if (withhold)
        knobs().debug |= DBG_WITHHOLD_FIRST_TILE;
    else
        knobs().debug &= ~DBG_WITHHOLD_FIRST_TILE;
    return RS_OK;
}

}  // extern "C"
