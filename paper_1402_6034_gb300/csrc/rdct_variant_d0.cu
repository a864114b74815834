// Instantiations of the variant kernel for anti-diagonal classes 0..4
// (split across translation units so they compile in parallel).
#include "rdct_variant.cuh"

namespace rdct {
template cudaError_t launch_variant_d<0>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<1>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<2>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<3>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<4>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
}  // namespace rdct
