// rs_sort64.cu -- scatter passes of 64-bit keys (K = 64, D = 8: eight
// passes), unsigned or typed, keys only or carrying 32-bit or 64-bit values.
#include "rs_internal.h"
#include "rs_onesweep_launch.cuh"

namespace rs {

namespace {

// Scatter-pass shapes of 64-bit keys: 384 threads x 7 keys (a tile of 2688)
// with no or 32-bit values, 384 x 6 (2304) with 64-bit values, two CTAs per
// SM, look-back window 8.  The shared-memory plan of a tile holds twice the
// key words of a 32-bit tile (and twice the value words), hence the shorter
// tiles.
constexpr int T64 = 384, B64 = 2, W64 = 8;

template <bool PAIRS, typename V, typename S, bool TYPED>
rs_status pass64(unsigned long long* ka, V* va, unsigned long long* kb, V* vb, uint32_t n,
                 uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status, void* status_clear,
                 uint32_t key_type, cudaStream_t stream) {
    constexpr int J = sizeof(V) == 8 ? kWideItems64V64 : kWideItems64;
    const SegView none{};
    return launch_onesweep_shape<T64, J, B64, W64, PAIRS, S, false, TYPED, unsigned long long, V>(
        ka, va, kb, vb, n, pass, pass, ctrl, sticky, status, status_clear, none, key_type, stream);
}

template <bool PAIRS, typename V, typename S>
rs_status pass64_typed(unsigned long long* ka, V* va, unsigned long long* kb, V* vb, uint32_t n,
                       uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status,
                       void* status_clear, uint32_t key_type, cudaStream_t stream) {
    if (key_type == KEY_U64)
        return pass64<PAIRS, V, S, false>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                          status_clear, KEY_U32, stream);
    // Typed keys: from typed_split_min items on, the passes that need no
    // maps run without them (see ROLE_PLAIN_PASSES) and both instances are
    // launched for every pass; below it the mapping instance runs them all.
    if (!typed_split(n))
        return pass64<PAIRS, V, S, true>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                         status_clear, key_type, stream);
    const rs_status st = pass64<PAIRS, V, S, false>(ka, va, kb, vb, n, pass, ctrl, sticky, status,
                                                    status_clear, key_type | ROLE_PLAIN_PASSES,
                                                    stream);
    if (st != RS_OK) return st;
    return pass64<PAIRS, V, S, true>(ka, va, kb, vb, n, pass, ctrl, sticky, status, status_clear,
                                     key_type | ROLE_MAP_PASSES, stream);
}

template <typename S>
rs_status pass64_values(unsigned long long* ka, void* va, unsigned long long* kb, void* vb,
                        uint32_t val_bytes, uint32_t n, uint32_t pass, Ctrl* ctrl,
                        uint32_t* sticky, void* status, void* status_clear, uint32_t key_type,
                        cudaStream_t stream) {
    switch (val_bytes) {
    case 0:
        return pass64_typed<false, uint32_t, S>(ka, nullptr, kb, nullptr, n, pass, ctrl, sticky,
                                                status, status_clear, key_type, stream);
    case 4:
        return pass64_typed<true, uint32_t, S>(ka, static_cast<uint32_t*>(va), kb,
                                               static_cast<uint32_t*>(vb), n, pass, ctrl, sticky,
                                               status, status_clear, key_type, stream);
    case 8:
        return pass64_typed<true, unsigned long long, S>(
            ka, static_cast<unsigned long long*>(va), kb, static_cast<unsigned long long*>(vb), n,
            pass, ctrl, sticky, status, status_clear, key_type, stream);
    default: return RS_ERR_INVALID_ARG;
    }
}

}  // namespace

rs_status launch_pass_k64(uint32_t key_type, uint32_t val_bytes, bool wide,
                          unsigned long long* ka, void* va, unsigned long long* kb, void* vb,
                          uint32_t n, uint32_t pass, Ctrl* ctrl, uint32_t* sticky, void* status,
                          void* status_clear, cudaStream_t stream) {
    if (key_type < KEY_U64 || key_type > KEY_F64) return RS_ERR_INVALID_ARG;
    return wide ? pass64_values<unsigned long long>(ka, va, kb, vb, val_bytes, n, pass, ctrl,
                                                    sticky, status, status_clear, key_type, stream)
                : pass64_values<uint32_t>(ka, va, kb, vb, val_bytes, n, pass, ctrl, sticky, status,
                                          status_clear, key_type, stream);
}

}  // namespace rs
