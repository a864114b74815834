// rdct_fused.cu -- dispatch of the fused path (Sec. 3 of Cintra & Bayer:
// forward, zonal truncation with the S scaling, inverse, squared error) and
// the persistent batch kernels.
#include "rdct_blocks.cuh"

namespace rdct {

cudaError_t launch_fused_single(const JobDesc &job, int kind, void *acc, unsigned long long *acc8, int ctas_per_sm,
                                int warps, cudaStream_t s) {
    if (kind == RDCT_KIND_RDCT && !job.dstf)
        return launch_fused2_single(job, reinterpret_cast<unsigned long long *>(acc), acc8, ctas_per_sm, 0, s);
    const int d = diag_class_host(job.r);
    const int64_t items = (int64_t)job.nbh * job.segs;
    // the 8-bit reconstruction is formed when it is stored or its error is wanted
    const int out = (job.dst || acc8 ? 1 : 0) | (job.dstf ? 2 : 0);
    const DctConsts C = kind == RDCT_KIND_DCT ? make_dct_consts() : DctConsts{};
#define RDCT_SINGLE(o, k) return launch_single_variant<o, k>(d, items, ctas_per_sm, warps, job, acc, acc8, C, s)
    if (kind == RDCT_KIND_RDCT) {
        switch (out) {
            case 0: RDCT_SINGLE(0, RDCT_KIND_RDCT);
            case 1: RDCT_SINGLE(1, RDCT_KIND_RDCT);
            case 2: RDCT_SINGLE(2, RDCT_KIND_RDCT);
            default: RDCT_SINGLE(3, RDCT_KIND_RDCT);
        }
    }
    switch (out) {
        case 0: RDCT_SINGLE(0, RDCT_KIND_DCT);
        case 1: RDCT_SINGLE(1, RDCT_KIND_DCT);
        case 2: RDCT_SINGLE(2, RDCT_KIND_DCT);
        default: RDCT_SINGLE(3, RDCT_KIND_DCT);
    }
#undef RDCT_SINGLE
}

int fused_class_of(int r, int blocks_per_thread) {
    return blocks_per_thread == 2 ? r - 1 : diag_class_host(r);
}

int batch_group_of_class(int cls, int blocks_per_thread) {
    if (blocks_per_thread == 2) return cls;
    return cls <= 5 ? 0 : (cls <= 8 ? 1 : 2);
}

cudaError_t launch_fused_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, unsigned long long *acc_u64,
                               unsigned long long *acc8, int group, int ctas_per_sm, int warps, int blocks_per_thread,
                               bool overlap, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    if (blocks_per_thread == 2)
        return launch_fused2_batch(jobs, chunks, nchunks, acc_u64, acc8, group + 1, ctas_per_sm, overlap, s);
    if (group == 0)
        launch_persistent(fused_batch_kernel<1, 0, 5>, nchunks, ctas_per_sm, warps, s, jobs, chunks, nchunks, acc_u64,
                          acc8);
    else if (group == 1)
        launch_persistent(fused_batch_kernel<1, 6, 8>, nchunks, ctas_per_sm, warps, s, jobs, chunks, nchunks, acc_u64,
                          acc8);
    else
        launch_persistent(fused_batch_kernel<1, 9, 14>, nchunks, ctas_per_sm, warps, s, jobs, chunks, nchunks, acc_u64,
                          acc8);
    return cudaGetLastError();
}

}  // namespace rdct
