// Batch launches of the fused kernel: one persistent launch per anti-diagonal
// class of r present in the batch (each class at its own register budget).
#include "rdct_fused2.cuh"

namespace rdct {

cudaError_t launch_fused2_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, unsigned long long *acc,
                                int d, int ctas_per_sm, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    Fused2Args a{};
    a.jobs = jobs;
    a.chunks = chunks;
    a.nchunks = nchunks;
    a.acc = acc;
    switch (d) {
#define RDCT_F2B(dd)                                                                                         \
    case dd:                                                                                                 \
        launch_staged(fused2_kernel<dd, dd, false, Fused2Shape<dd>::threads, Fused2Shape<dd>::min_blocks>,     \
                      nchunks, ctas_per_sm, Fused2Shape<dd>::threads / 32, kFused2MaxCtas, kFused2Smem, s, a); \
        break;
        RDCT_F2B(0) RDCT_F2B(1) RDCT_F2B(2) RDCT_F2B(3) RDCT_F2B(4) RDCT_F2B(5) RDCT_F2B(6) RDCT_F2B(7)
        RDCT_F2B(8) RDCT_F2B(9) RDCT_F2B(10) RDCT_F2B(11) RDCT_F2B(12) RDCT_F2B(13) RDCT_F2B(14)
#undef RDCT_F2B
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rdct
