// rs_pipeline.cu -- host launcher of k_onesweep_ws, the warp-specialised
// scatter pass of 32-bit keys with 32-bit values (rs_pipeline.cuh).
#include "rs_internal.h"
#include "rs_pipeline.cuh"

namespace rs {

namespace {
// Teams (warps): rank, count, look-back, store; items per rank-warp lane.
constexpr int kRW = 12, kCW = 4, kLW = 4, kSW = 4, kItems = 14, kWindow = 6;
using Shape = PipeShape<kRW, kCW, kLW, kSW, kItems>;
}  // namespace

uint32_t pipeline_tile() { return Shape::TILE; }

rs_status launch_pipeline_pairs(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb,
                                uint32_t n, uint32_t pass, uint32_t slot, Ctrl* ctrl,
                                uint32_t* sticky, void* status, void* status_clear,
                                cudaStream_t stream) {
    auto kern = k_onesweep_ws<kRW, kCW, kLW, kSW, kItems, kWindow>;
    static DeviceOnce smem_set;
    rs_status st = allow_smem_once(kern, Shape::BYTES, smem_set);
    if (st != RS_OK) return st;
    DeviceInfo di;
    st = device_info(&di);
    if (st != RS_OK) return st;
    const uint32_t tiles = (uint32_t)((n + (size_t)Shape::TILE - 1) / Shape::TILE);
    uint32_t grid = (uint32_t)di.sm_count;  // one CTA per SM
    if (grid > tiles) grid = tiles;
    if (grid == 0) return RS_OK;
    note_launch_begin(KK_ONESWEEP, stream);
    kern<<<grid, Shape::THREADS, Shape::BYTES, stream>>>(
        ka, va, kb, vb, n, pass, slot, tiles, ctrl, sticky, static_cast<uint32_t*>(status),
        static_cast<uint32_t*>(status_clear), tiles * RADIX, knobs().spin_limit, knobs().debug);
    note_launch_end(KK_ONESWEEP, stream);
    return cudaPeekAtLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

}  // namespace rs
