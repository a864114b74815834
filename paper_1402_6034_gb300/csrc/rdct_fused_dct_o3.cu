// Instantiates the single-plane fused kernels for transform kind DCT and
// output mode 3 (bit 0: uint8 reconstruction, bit 1: FP32 reconstruction).
#include "rdct_fused_single.cuh"

namespace rdct {
template cudaError_t launch_single_variant<3, 1>(int, int64_t, int, int, const JobDesc &, void *,
                                                      unsigned long long *,
                                                      const DctConsts &, cudaStream_t);
}  // namespace rdct
