// Launch of the RDCT pass of the r sweep (see rdct_sweep2.cuh) and the
// on-device construction of the sweep's job and chunk tables (both passes).
#include <algorithm>

#include "rdct_sweep2.cuh"

namespace rdct {

cudaError_t launch_sweep2(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, double *out, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    Fused2Args a{};
    a.jobs = jobs;
    a.chunks = chunks;
    a.nchunks = nchunks;
    // a programmatic dependent of the table builder: its launch overlaps the builder's tail
    return launch_staged(sweep2_kernel, nchunks, 0, 4, kFused2MaxCtas, kFused2Smem, true, s, a, out);
}

namespace {

__device__ int align_class(const void *p, int64_t pitch) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if ((a % 16) == 0 && (pitch % 16) == 0) return 16;
    if ((a % 8) == 0 && (pitch % 8) == 0) return 8;
    return 1;
}

// Up to kSweepBuildBatch planes, passed by value so that building the tables
// needs no host-to-device copy (and no stream synchronisation); base[i] is the
// index of plane i's first chunk, or with `tiles` set its first tile of 128
// blocks (host prefix sums).
struct PlaneBatch {
    rdct_plane p[kSweepBuildBatch];
    int32_t base[kSweepBuildBatch];
    int32_t first, n, tiles;
};
// kernel parameters: the batch and three pointers, within the 32764-byte limit
static_assert(sizeof(PlaneBatch) + 3 * sizeof(void *) <= 32764, "sweep table batch too large for kernel parameters");

// One warp per plane: every lane reads the same descriptor (a broadcast from
// the parameter bank), lane 0 writes the job, and the lanes clear its 64
// output bins and write the plane's chunks (runs of at most kSweepChunkStrips
// items of 32 column pairs) -- or, for the tiled pass, only the job, with its
// first tile in JobDesc::pad.
__global__ void __launch_bounds__(32) build_sweep_tables_kernel(const PlaneBatch b, JobDesc *jobs, Chunk *chunks,
                                                                double *out) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int i = blockIdx.x;
    const int lane = threadIdx.x;
    out[(int64_t)(b.first + i) * 64 + lane] = 0.0;
    out[(int64_t)(b.first + i) * 64 + 32 + lane] = 0.0;
    const rdct_plane pl = b.p[i];
    JobDesc j{};
    j.src = pl.ptr;
    j.src_pitch = pl.pitch;
    j.nbw = pl.w / 8;
    j.nbh = pl.h / 8;
    j.r = 64;
    j.image = b.first + i;
    j.segs = (j.nbw + 31) / 32;
    j.align = align_class(pl.ptr, pl.pitch);
    j.dalign = 16;
    j.pad = b.tiles ? b.base[i] : 0;
    if (lane == 0) jobs[b.first + i] = j;
    if (b.tiles) return;
    const int32_t items = fused_items_of(j);
    const int32_t nch = (items + kSweepChunkStrips - 1) / kSweepChunkStrips;
    for (int32_t t = lane; t < nch; t += 32) {
        const int32_t it = t * kSweepChunkStrips;
        chunks[b.base[i] + t] = Chunk{b.first + i, it, items - it < kSweepChunkStrips ? items - it : kSweepChunkStrips, 0};
    }
}

}  // namespace

int64_t sweep_chunk_count(const rdct_plane &p) {
    const int64_t pairs = (int64_t)((p.h / 8 + kFusedVRows - 1) / kFusedVRows) * (p.w / 8);
    const int64_t items = (pairs + 31) / 32;
    return (items + kSweepChunkStrips - 1) / kSweepChunkStrips;
}

cudaError_t build_sweep_tables(const rdct_plane *planes, int32_t n, bool tiles, JobDesc *jobs, Chunk *chunks,
                               double *out, cudaStream_t s) {
    int32_t base = 0;
    for (int32_t first = 0; first < n; first += kSweepBuildBatch) {
        PlaneBatch b;
        b.first = first;
        b.n = std::min(kSweepBuildBatch, n - first);
        b.tiles = tiles ? 1 : 0;
        for (int32_t i = 0; i < b.n; ++i) {
            b.p[i] = planes[first + i];
            b.base[i] = base;
            base += (int32_t)(tiles ? sweep_tiles_of(planes[first + i]) : sweep_chunk_count(planes[first + i]));
        }
        build_sweep_tables_kernel<<<b.n, 32, 0, s>>>(b, jobs, chunks, out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace rdct
