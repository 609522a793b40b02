// rs_onesweep_pairs.cu -- scatter passes of the key-value sorts.
#include "rs_onesweep_launch.cuh"

namespace rs {

rs_status launch_onesweep_pairs(int cfg, bool wide, uint32_t* ka, uint32_t* va, uint32_t* kb,
                                uint32_t* vb, uint32_t n, uint32_t pass, uint32_t slot,
                                Ctrl* ctrl, uint32_t* sticky, void* status, void* status_clear,
                                const SegView* seg, uint32_t key_type, cudaStream_t stream) {
    const SegView none{};
    if (seg != nullptr)  // segment prefixes stay below 2^30: 32-bit status words
        return launch_onesweep_variant<true, uint32_t, true>(cfg, ka, va, kb, vb, n, pass, slot,
                                                             ctrl, sticky, status, status_clear,
                                                             *seg, key_type, stream);
    if (wide)
        return launch_onesweep_variant<true, unsigned long long, false>(
            cfg, ka, va, kb, vb, n, pass, slot, ctrl, sticky, status, status_clear, none,
            key_type, stream);
    return launch_onesweep_variant<true, uint32_t, false>(cfg, ka, va, kb, vb, n, pass, slot,
                                                          ctrl, sticky, status, status_clear,
                                                          none, key_type, stream);
}

}  // namespace rs
