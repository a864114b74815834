// Instantiations of the variant kernel for anti-diagonal classes 10..14
// (split across translation units so they compile in parallel).
#include "rdct_variant.cuh"

namespace rdct {
template cudaError_t launch_variant_d<10>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<11>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<12>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<13>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
template cudaError_t launch_variant_d<14>(const JobDesc &, const MatConsts &, double *, cudaStream_t);
}  // namespace rdct
