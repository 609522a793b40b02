// rs_noalloc.cu -- rs_sort_pairs_noalloc: the sort without any device
// allocation, for callers that must not allocate device memory at call time.
//
// Its scratch (control block, look-back status words and the alternate key
// and value buffers) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads this library holds until the process exits.
#include <mutex>

#include "rs_internal.h"

namespace {

constexpr size_t kMaxItems = RS_NOALLOC_MAX_ITEMS;
// Enough for the workspace of kMaxItems key-value pairs (8.51 MiB: two
// 4 MiB alternate buffers, two 256 KiB status arrays, the control block).
constexpr size_t kScratchBytes = size_t(9) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_on[64] = {nullptr};  // device address of the array, per device

}  // namespace

extern "C" rs_status rs_sort_pairs_noalloc(uint32_t* d_keys, uint32_t* d_vals, size_t n,
                                           void* cuda_stream) {
    if (n > kMaxItems) return RS_ERR_UNSUPPORTED;
    rs_status st = rs::check_sort_args(d_keys, d_vals, n);
    if (st != RS_OK || n == 0) return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RS_ERR_CUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_scratch_on[dev] == nullptr) {
            // The array's name is a host-side stand-in; its address on this
            // device (the current one) is looked up once and cached.
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
                // Clear the runtime's last error, so that a later, unrelated
                // launch check does not report this failure as its own.
                (void)cudaGetLastError();
                return RS_ERR_CUDA;
            }
            g_scratch_on[dev] = p;
        }
        scratch = g_scratch_on[dev];
    }
    if (rs::layout_for(n, d_vals != nullptr).total > kScratchBytes) return RS_ERR_UNSUPPORTED;
    // enqueue_sort zeroes the control block and clears the first status
    // array itself, so whatever an earlier call left in the array is harmless.
    return rs::enqueue_sort(d_keys, d_vals, (uint32_t)n, static_cast<cudaStream_t>(cuda_stream),
                            scratch, kScratchBytes);
}
