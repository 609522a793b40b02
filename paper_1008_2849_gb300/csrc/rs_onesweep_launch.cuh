// rs_onesweep_launch.cuh -- host launcher of k_onesweep for every tile shape
// of kTileConfigs; included once per value flavour (keys / pairs).
#pragma once

#include "rs_internal.h"
#include "rs_onesweep.cuh"

namespace rs {

template <int THREADS, int ITEMS, bool PAIRS, typename S>
static rs_status launch_onesweep_shape(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb,
                                       uint32_t n, uint32_t pass, Ctrl* ctrl, uint32_t* sticky,
                                       void* status, void* status_clear, cudaStream_t stream) {
    constexpr uint32_t TILE = THREADS * ITEMS;
    const size_t smem = TILE * sizeof(uint32_t);
    auto kern = k_onesweep<THREADS, ITEMS, PAIRS, S>;
    static uint64_t attr_set_on = 0;  // one bit per device that has the attribute
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return RS_ERR_CUDA;
    if (!((attr_set_on >> dev) & 1u)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return RS_ERR_CUDA;
        attr_set_on |= 1ull << dev;
    }
    const uint32_t tiles = (uint32_t)((n + (size_t)TILE - 1) / TILE);
    note_launch_begin(KK_ONESWEEP, stream);
    kern<<<tiles, THREADS, smem, stream>>>(ka, va, kb, vb, n, pass, ctrl, sticky,
                                           static_cast<S*>(status), static_cast<S*>(status_clear),
                                           knobs().spin_limit, knobs().debug);
    note_launch_end(KK_ONESWEEP, stream);
    return cudaPeekAtLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

template <bool PAIRS, typename S>
static rs_status launch_onesweep_typed(int cfg, uint32_t* ka, uint32_t* va, uint32_t* kb,
                                       uint32_t* vb, uint32_t n, uint32_t pass, Ctrl* ctrl,
                                       uint32_t* sticky, void* status, void* status_clear,
                                       cudaStream_t stream) {
    switch (cfg) {
    case 0: return launch_onesweep_shape<256, 16, PAIRS, S>(ka, va, kb, vb, n, pass, ctrl, sticky, status, status_clear, stream);
    case 1: return launch_onesweep_shape<512, 16, PAIRS, S>(ka, va, kb, vb, n, pass, ctrl, sticky, status, status_clear, stream);
    case 2: return launch_onesweep_shape<512, 12, PAIRS, S>(ka, va, kb, vb, n, pass, ctrl, sticky, status, status_clear, stream);
    default: return RS_ERR_INVALID_ARG;
    }
}

}  // namespace rs
