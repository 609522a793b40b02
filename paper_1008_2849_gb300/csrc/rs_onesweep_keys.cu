// rs_onesweep_keys.cu -- scatter passes of the keys-only sort.
#include "rs_onesweep_launch.cuh"

namespace rs {

rs_status launch_onesweep_keys(int cfg, bool wide, uint32_t* ka, uint32_t* kb, uint32_t n,
                               uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status,
                               void* status_clear, cudaStream_t stream) {
    if (wide)
        return launch_onesweep_typed<false, unsigned long long>(cfg, ka, nullptr, kb, nullptr, n, pass,
                                                                ctrl, sticky, status, status_clear, stream);
    return launch_onesweep_typed<false, uint32_t>(cfg, ka, nullptr, kb, nullptr, n, pass, ctrl,
                                                  sticky, status, status_clear, stream);
}

}  // namespace rs
