// rs_onesweep_keys.cu -- scatter passes of the keys-only sorts.
#include "rs_onesweep_launch.cuh"

namespace rs {

rs_status launch_onesweep_keys(int cfg, bool wide, uint32_t* ka, uint32_t* kb, uint32_t n,
                               uint32_t pass, uint32_t slot, Ctrl* ctrl, uint32_t* sticky,
                               void* status, void* status_clear, const SegView* seg,
                               uint32_t key_type, cudaStream_t stream) {
    const SegView none{};
    if (seg != nullptr)  // segment prefixes stay below 2^30: 32-bit status words
        return launch_onesweep_variant<false, uint32_t, true>(
            cfg, ka, nullptr, kb, nullptr, n, pass, slot, ctrl, sticky, status, status_clear,
            *seg, key_type, stream);
    if (wide)
        return launch_onesweep_variant<false, unsigned long long, false>(
            cfg, ka, nullptr, kb, nullptr, n, pass, slot, ctrl, sticky, status, status_clear,
            none, key_type, stream);
    return launch_onesweep_variant<false, uint32_t, false>(
        cfg, ka, nullptr, kb, nullptr, n, pass, slot, ctrl, sticky, status, status_clear, none,
        key_type, stream);
}

}  // namespace rs
