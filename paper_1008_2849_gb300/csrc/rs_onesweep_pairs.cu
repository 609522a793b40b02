// rs_onesweep_pairs.cu -- scatter passes of the key-value sort.
#include "rs_onesweep_launch.cuh"

namespace rs {

rs_status launch_onesweep_pairs(int cfg, bool wide, uint32_t* ka, uint32_t* va, uint32_t* kb,
                                uint32_t* vb, uint32_t n, uint32_t pass, Ctrl* ctrl,
                                uint32_t* sticky, void* status, void* status_clear,
                                cudaStream_t stream) {
    if (wide)
        return launch_onesweep_typed<true, unsigned long long>(cfg, ka, va, kb, vb, n, pass, ctrl,
                                                               sticky, status, status_clear, stream);
    return launch_onesweep_typed<true, uint32_t>(cfg, ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                                 status_clear, stream);
}

}  // namespace rs
