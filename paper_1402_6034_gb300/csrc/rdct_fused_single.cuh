// rdct_fused_single.cuh -- definition of the single-plane fused launch
// (instantiated once per output mode and transform kind in its own
// translation unit so that the 15 anti-diagonal specialisations of each
// compile in parallel).
#pragma once
#include "rdct_blocks.cuh"

namespace rdct {

template <int OUT, int KIND>
cudaError_t launch_single_variant(int d, int64_t items, int ctas_per_sm, int warps, const JobDesc &job, void *acc,
                                  unsigned long long *acc8, const DctConsts &C, cudaStream_t s) {
    switch (d) {
#define RDCT_LCASE(dd)                                                                                      \
    case dd:                                                                                                \
        launch_persistent(fused_single_kernel<dd, OUT, KIND>, items, ctas_per_sm, warps, s, job, acc, acc8, C); \
        break;
        RDCT_LCASE(0) RDCT_LCASE(1) RDCT_LCASE(2) RDCT_LCASE(3) RDCT_LCASE(4) RDCT_LCASE(5) RDCT_LCASE(6)
        RDCT_LCASE(7) RDCT_LCASE(8) RDCT_LCASE(9) RDCT_LCASE(10) RDCT_LCASE(11) RDCT_LCASE(12) RDCT_LCASE(13)
        RDCT_LCASE(14)
#undef RDCT_LCASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rdct
