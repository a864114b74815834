// Single-plane launches of the fused kernel (one anti-diagonal class each).
#include <algorithm>

#include "rdct_fused2.cuh"

namespace rdct {

cudaError_t launch_fused2_single(const JobDesc &job, unsigned long long *acc, int ctas_per_sm, int chunk_items,
                                 cudaStream_t s) {
    Fused2Args a{};
    a.single = job;
    const int64_t items = fused_items_of(job);
    if (chunk_items <= 0) {  // enough chunks for every resident warp, at most 16 strips each
        const int64_t warps = (int64_t)sm_count() * 16;
        chunk_items = (int)std::min<int64_t>(16, std::max<int64_t>(1, items / warps));
    }
    a.chunk_items = chunk_items;
    a.nchunks = (int32_t)((items + a.chunk_items - 1) / a.chunk_items);
    a.acc = acc;
    if (a.nchunks == 0) return cudaSuccess;
    switch (diag_class(job.r)) {
#define RDCT_F2(d)                                                                                          \
    case d:                                                                                                 \
        launch_staged(fused2_kernel<d, d, true, Fused2Shape<d>::threads, Fused2Shape<d>::min_blocks>,       \
                      a.nchunks, ctas_per_sm, Fused2Shape<d>::threads / 32, kFused2MaxCtas, kFused2Smem, s, a); \
        break;
        RDCT_F2(0) RDCT_F2(1) RDCT_F2(2) RDCT_F2(3) RDCT_F2(4) RDCT_F2(5) RDCT_F2(6) RDCT_F2(7)
        RDCT_F2(8) RDCT_F2(9) RDCT_F2(10) RDCT_F2(11) RDCT_F2(12) RDCT_F2(13) RDCT_F2(14)
#undef RDCT_F2
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rdct
