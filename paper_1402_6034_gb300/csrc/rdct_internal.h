// rdct_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/rdct.h"

namespace rdct {

// One plane as the kernels see it (device descriptor).
struct JobDesc {
    const uint8_t *src;
    uint8_t *dst;     // uint8 reconstruction or nullptr
    float *dstf;      // FP32 reconstruction or nullptr
    int64_t src_pitch, dst_pitch, dstf_pitch;  // bytes, bytes, floats
    int32_t nbw, nbh; // blocks per row / per column
    int32_t r;        // retained coefficients, 1..64
    int32_t image;    // SSE slot
    int32_t segs;     // strips per block row = ceil(nbw / (32 * blocks_per_thread))
    int32_t align;    // 16 if src and src_pitch are 16-byte aligned, 8 if 8-byte, else 1
    int32_t dalign;   // same for dst
    int32_t pad;
};

// The fused kernel's work items: a thread owns kFusedVRows vertically adjacent
// blocks (a "column pair" of one row pair); the row pairs x columns of a plane
// are numbered row-major and an item is a run of 32 consecutive column pairs
// (one per lane), which may wrap into the next row pair, so no lane idles at
// the end of a row.  The scalar kernel's items are one block row by 32 blocks.
constexpr int kFusedVRows = 2;
__host__ __device__ inline int32_t fused_items_of(const JobDesc &j) {
    const int64_t pairs = (int64_t)((j.nbh + kFusedVRows - 1) / kFusedVRows) * j.nbw;
    return (int32_t)((pairs + 31) / 32);
}
__host__ __device__ inline int32_t strips_of(const JobDesc &j, int vrows) {
    return vrows == kFusedVRows ? fused_items_of(j) : j.nbh * j.segs;
}

// A run of consecutive strips of one job handed to one warp.  cls is the
// launch class of the job's r (fused_class_of): r - 1 for the two-block
// kernel, the anti-diagonal class of r for the scalar kernel.
struct Chunk {
    int32_t job, item0, nitems, cls;
};

// FP32 constants of the exact DCT (host-computed from cos in double).
struct DctConsts {
    float c[64];  // C[k][n]
};
// FP32 d_i d_j products (orthonormal scaling of C0 coefficients).
struct ScaleConsts {
    float dd[64];
};
// Forward and reconstruction matrices of the other transforms (signed DCT,
// floor / ceiling variants): a block A goes to F A F^T and back as G Yhat G^T.
struct MatConsts {
    float f[64];  // F, row-major
    float g[64];  // G, row-major
};
template <int D>
cudaError_t launch_variant_d(const JobDesc &job, const MatConsts &M, double *acc, cudaStream_t s);
// F and G of a variant in double (host); RDCT_ERR_ARG for floor(2C) (singular).
rdct_status variant_matrices(rdct_variant v, double F[8][8], double G[8][8]);

// Error state (thread-local message).
rdct_status set_error(rdct_status s, const std::string &msg);
rdct_status cuda_error(cudaError_t e, const char *what);
#define RDCT_CUDA_TRY(expr)                                        \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return ::rdct::cuda_error(e_, #expr); \
    } while (0)

DctConsts make_dct_consts();
ScaleConsts make_scale_consts();
int sm_count();
rdct_status validate_plane(const rdct_plane *p, const char *what);
JobDesc make_job(const rdct_plane &src, uint8_t *dst, int64_t dst_pitch, float *dstf, int64_t dstf_pitch, int32_t r,
                 int32_t image, int bpt);
int diag_class_host(int r);

// ---------------------------------------------------------------- launchers
// (all asynchronous on `s`; return cudaGetLastError of the launch)
cudaError_t launch_forward(const JobDesc &job, int32_t *Y, cudaStream_t s);
cudaError_t launch_forward_f32(const JobDesc &job, int kind, float *Y, cudaStream_t s);
cudaError_t launch_compress(const int32_t *Y, int64_t nblocks, int32_t r, float *Yc, cudaStream_t s);
cudaError_t launch_inverse(const float *Yc, int64_t nbw, int64_t nbh, int32_t r, int kind, uint8_t *u8,
                           int64_t pitch, float *f32, int64_t pitch_f32, cudaStream_t s);
// SSE of rec vs ref accumulated into acc[0] (uint64, u8 rec) or acc as double (f32 rec).
cudaError_t launch_sse(const JobDesc &ref, const uint8_t *rec_u8, int64_t rec_pitch, const float *rec_f32,
                       int64_t rec_pitch_f32, unsigned long long *acc_u64, double *acc_f64, cudaStream_t s);
cudaError_t launch_mse_finalize(const unsigned long long *acc_u64, const double *acc_f64, int use_u64,
                                double nsamples, double *mse, double *psnr, cudaStream_t s);
// Fused path for one job: acc is the caller's SSE slot (zeroed by the caller),
// used as uint64 576*SSE for kind RDCT and as double SSE for kind DCT; acc8
// (uint64, zeroed by the caller, or nullptr) receives the squared error of the
// 8-bit reconstruction, which is then formed even when job.dst is nullptr.
cudaError_t launch_fused_single(const JobDesc &job, int kind, void *acc, unsigned long long *acc8, int ctas_per_sm,
                                int warps, cudaStream_t s);
// Persistent batch kernels.  Chunks are grouped: with blocks_per_thread 2
// one group per r (64 groups, a kernel specialised for each r), with
// blocks_per_thread 1 one group per register class (3 groups).
// acc_u64[image] += 576 * SSE, and acc8[image] (unless nullptr) += the
// squared error of the 8-bit reconstruction.  ctas_per_sm <= 0 uses the
// occupancy limit.
constexpr int kBatchGroups = 64;
int fused_class_of(int r, int blocks_per_thread);
int batch_group_of_class(int cls, int blocks_per_thread);
// blocks_per_thread 2 selects the dp4a/f32x2 kernel (128 threads per CTA,
// strips of kFusedVRows block rows), 1 the scalar kernel with `warps` warps.
// overlap (blocks_per_thread 2): the launch may start while the previous
// launch of the same batch in the stream drains (programmatic dependent
// launch); pass false for the first launch of a batch.
cudaError_t launch_fused_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, unsigned long long *acc_u64,
                               unsigned long long *acc8, int group, int ctas_per_sm, int warps, int blocks_per_thread,
                               bool overlap, cudaStream_t s);
// The fused kernel for sm_103a issue rates (dp4a row pass, f32x2 inverse,
// cp.async ring): uint8 output or error only, any alignment.
cudaError_t launch_fused2_single(const JobDesc &job, unsigned long long *acc, unsigned long long *acc8,
                                 int ctas_per_sm, int chunk_items, cudaStream_t s);
cudaError_t launch_fused2_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, unsigned long long *acc,
                                unsigned long long *acc8, int r, int ctas_per_sm, bool overlap, cudaStream_t s);
// The same kernel with TMA loads and stores, for batch tables whose items are
// row pair x 32-column segments (tma_items_of) and whose planes have encoded
// tensor maps (two of kTensorMapBytes each per plane, see tma_encode_plane).
cudaError_t launch_fused2_tma_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks,
                                    const unsigned char *maps, unsigned long long *acc, unsigned long long *acc8,
                                    int r, int ctas_per_sm, bool overlap, cudaStream_t s);
inline int32_t tma_items_of(const JobDesc &j) { return ((j.nbh + 1) / 2) * ((j.nbw + 31) / 32); }
constexpr int kTensorMapBytes = 128;  // one encoded 2-D tensor map per plane (64-byte aligned in the table)
// TMA staging needs the source plane and the reconstruction (if any) to start
// on 16-byte boundaries with 16-byte multiple pitches, and the driver's
// tensor-map encoder.  tma_encode_plane writes the source's map and then the
// reconstruction's (zeros when there is none) into 2 * kTensorMapBytes.
bool tma_available();
bool tma_plane_ok(const JobDesc &j);
bool tma_encode_plane(const JobDesc &j, unsigned char *maps256);
// TMA-staged kernels bound their waits for a staged box; a warp whose wait
// runs out counts it and stops.  Each translation unit that instantiates
// those kernels holds its own counter; these read and clear them.
unsigned int take_tma_timeouts_r0();
unsigned int take_tma_timeouts_r1();
unsigned int take_tma_timeouts_r2();
unsigned int take_tma_timeouts_r3();
unsigned int take_tma_timeouts_r4();
unsigned int take_tma_timeouts_r5();
unsigned int take_tma_timeouts_r6();
unsigned int take_tma_timeouts_r7();
unsigned int take_tma_timeouts_r8();
unsigned int take_tma_timeouts_r9();
unsigned int take_tma_timeouts_r10();
unsigned int take_tma_timeouts_r11();
unsigned int take_tma_timeouts_r12();
unsigned int take_tma_timeouts_r13();
unsigned int take_tma_timeouts_r14();
unsigned int take_tma_timeouts_r15();
// In-place conversion of n uint64 576*SSE slots to double SSE (slots not
// nullptr), and of n uint64 squared errors of 8-bit reconstructions in slots8
// (if not nullptr) to double.
cudaError_t launch_sse576_to_double(void *slots, int32_t n, cudaStream_t s, void *slots8 = nullptr);
// Sweep: per-plane zigzag energy, then suffix sums into SSE(r).  The RDCT
// pass runs over chunks: runs of at most kSweepChunkStrips strips of
// kFusedVRows block rows.
constexpr int kSweepChunkStrips = 8;
cudaError_t launch_sweep2(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, double *out, cudaStream_t s);
// Sweep tables built on the device from plane descriptors passed as kernel
// parameters (batches of kSweepBuildBatch planes; no host-to-device copy):
// the jobs and the chunks of the per-block pass, or with `tiles` the jobs of
// the tiled pass alone (each with its first tile).
constexpr int kSweepBuildBatch = 1024;
int64_t sweep_chunk_count(const rdct_plane &p);
// (also clears out: the planes' 64 bins each)
cudaError_t build_sweep_tables(const rdct_plane *planes, int32_t n, bool tiles, JobDesc *jobs, Chunk *chunks,
                               double *out, cudaStream_t s);
// whether the sweep of this kind runs tiled (the DCT pass on the tensor cores)
inline bool sweep_is_tiled(int kind) { return kind == RDCT_KIND_DCT; }
cudaError_t launch_sweep(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, int kind, double *out,
                         int32_t nplanes, int32_t ntiles, cudaStream_t s);
// The DCT pass of the sweep on the tensor cores (rdct_sweep_tc.cu): tiles of
// 128 blocks of one plane, JobDesc::pad = the plane's first tile.
constexpr int kSweepTileBlocks = 128;
__host__ __device__ inline int64_t sweep_tiles_of(const rdct_plane &p) {
    return ((int64_t)(p.w / 8) * (p.h / 8) + kSweepTileBlocks - 1) / kSweepTileBlocks;
}
cudaError_t launch_sweep_dct_tc(const JobDesc *jobs, int32_t nplanes, int32_t total_tiles, double *out,
                                cudaStream_t s);
unsigned int take_sweep_tc_timeouts();
cudaError_t launch_sweep_finalize(double *out, int32_t nplanes, int kind, cudaStream_t s);
// 2-D copy of w bytes by h rows done by a kernel (for pageable host memory the
// device addresses through the host page tables).
cudaError_t launch_copy2d(void *dst, int64_t dpitch, const void *src, int64_t spitch, int32_t w, int32_t h,
                          cudaStream_t s);
// True when the current device reads and writes pageable host memory through
// the host's page tables.
bool device_pageable_access(int device);
// True when every byte of [p, p + bytes) is plain (pageable) host memory that
// CUDA does not know (first and last byte checked).
bool is_pageable_host(const void *p, int64_t bytes);

}  // namespace rdct
