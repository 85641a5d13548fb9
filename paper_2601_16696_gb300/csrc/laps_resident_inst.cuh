// laps_resident_inst.cuh -- instantiates the resident kernel for one target
// (LAPS_INST_KIND) over the supported (lanes per chain, coordinates per lane)
// shapes, with and without the full-rank bias proxy, and defines its host-side launch / occupancy dispatchers.  Each
// target lives in its own translation unit so the shapes compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "laps_resident_kernel.cuh"

#ifndef LAPS_INST_KIND
#error "define LAPS_INST_KIND before including laps_resident_inst.cuh"
#endif

#define LAPS_SHAPES(X) \
    X(4, 4)            \
    X(8, 4)            \
    X(8, 8)            \
    X(16, 4)           \
    X(16, 8)           \
    X(32, 4)           \
    X(32, 8)           \
    X(32, 16)

namespace laps {

template <int KIND>
struct ResidentDispatch {
    static const void* fn(int lpc, int cpl, bool fr) {
#define LAPS_FN(L, C)                                                                            \
    if (lpc == L && cpl == C) {                                                                  \
        if constexpr (KIND == TGT_GAUSS_DENSE) /* no full-rank form */                           \
            return fr ? nullptr : reinterpret_cast<const void*>(&laps_resident_kernel<KIND, L, C, false>); \
        else                                                                                     \
            return fr ? reinterpret_cast<const void*>(&laps_resident_kernel<KIND, L, C, true>)   \
                      : reinterpret_cast<const void*>(&laps_resident_kernel<KIND, L, C, false>); \
    }
        LAPS_SHAPES(LAPS_FN)
#undef LAPS_FN
        return nullptr;
    }
};

#define LAPS_CAT2(a, b) a##b
#define LAPS_CAT(a, b) LAPS_CAT2(a, b)

// returns the kernel symbol for (lpc, cpl), with the full-rank proxy's block
// products when fr, or nullptr if not built
const void* LAPS_CAT(resident_kernel_, LAPS_INST_KIND)(int lpc, int cpl, bool fr) {
    return ResidentDispatch<LAPS_INST_KIND>::fn(lpc, cpl, fr);
}

}  // namespace laps
