// Instantiations of the fused kernel for r = 9..16 (eight per translation
// unit so that the 64 specialisations compile in parallel).
#include "rdct_fused2.cuh"

namespace rdct {
template cudaError_t launch_fused2_r<9>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<10>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<11>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<12>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<13>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<14>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<15>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<16>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<9>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<10>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<11>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<12>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<13>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<14>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<15>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<16>(const TmaArgs &, int, bool, cudaStream_t);
}  // namespace rdct
