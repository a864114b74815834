// Instantiates the single-plane fused kernels for transform kind RDCT and
// output mode 1 (bit 0: uint8 reconstruction, bit 1: FP32 reconstruction).
#include "rdct_fused_single.cuh"

namespace rdct {
template cudaError_t launch_single_variant<1, 0>(int, int64_t, int, int, const JobDesc &, void *,
                                                      unsigned long long *,
                                                      const DctConsts &, cudaStream_t);
}  // namespace rdct
