// Instantiations of the fused kernel for r = 21..24 (four per translation unit
// so that the 64 specialisations, each with and without the 8-bit error, compile
// in parallel).
#include "rdct_fused2.cuh"

namespace rdct {
template cudaError_t launch_fused2_r<21>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<22>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<23>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<24>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<21>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<22>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<23>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<24>(const TmaArgs &, int, bool, cudaStream_t);

// Reads and clears this translation unit's count of TMA waits that ran out
// (each translation unit holds its own copy of the counter).
unsigned int take_tma_timeouts_r5() {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tma_timeouts, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_tma_timeouts, &zero, sizeof(zero));
    }
    return v;
}
}  // namespace rdct
