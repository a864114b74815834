// Instantiations of the fused kernel for r = 57..60 (four per translation unit
// so that the 64 specialisations, each with and without the 8-bit error, compile
// in parallel).
#include "rdct_fused2.cuh"

namespace rdct {
template cudaError_t launch_fused2_r<57>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<58>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<59>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<60>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<57>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<58>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<59>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<60>(const TmaArgs &, int, bool, cudaStream_t);

// Reads and clears this translation unit's count of TMA waits that ran out
// (each translation unit holds its own copy of the counter).
unsigned int take_tma_timeouts_r14() {
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
