// Instantiations of the variant kernel for anti-diagonal classes 5..9
// (split across translation units so they compile in parallel).
#include "rdct_variant.cuh"

namespace rdct {
template cudaError_t launch_variant_d<5>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<6>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<7>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<8>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<9>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
}  // namespace rdct
