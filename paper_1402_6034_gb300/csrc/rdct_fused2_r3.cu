// Instantiations of the fused kernel for r = 25..32 (eight per translation
// unit so that the 64 specialisations compile in parallel).
#include "rdct_fused2.cuh"

namespace rdct {
template cudaError_t launch_fused2_r<25>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<26>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<27>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<28>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<29>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<30>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<31>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_r<32>(const Fused2Args &, bool, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<25>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<26>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<27>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<28>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<29>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<30>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<31>(const TmaArgs &, int, bool, cudaStream_t);
template cudaError_t launch_fused2_tma_r<32>(const TmaArgs &, int, bool, cudaStream_t);
}  // namespace rdct
