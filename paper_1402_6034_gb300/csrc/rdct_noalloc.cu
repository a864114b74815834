// rdct_noalloc.cu -- rdct_sweep_noalloc: the r sweep without any allocation.
//
// Some callers cannot allocate device memory at the moment they call us: a
// host framework that owns the whole device heap through its own allocator
// (where a stray cudaMalloc or cudaMallocAsync would fragment its pool or
// break its memory cap), a real-time loop in which an allocation could stall
// or synchronise the device, or a plug-in whose host process forbids device
// allocation outright.  rdct_sweep builds per-call descriptor tables in a
// stream-ordered allocation; this variant keeps them in one fixed device array
// that is part of the library image instead; both build them on the device
// from plane descriptors passed as kernel parameters and run the same kernels.  Nothing is allocated, on the device or on
// the host, on the success path.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocScratchBytes, 672 KiB) until the process
// exits.  In host code its name is only a host-side stand-in for the device
// variable, not a device address, so its device address is looked up with
// cudaGetSymbolAddress, once per device, with that device current, the first
// time the entry point runs on that device.  That first call should therefore
// come before any stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "rdct_device.cuh"
#include "rdct_internal.h"

namespace rdct {
namespace {

constexpr int32_t kNoAllocMaxPlanes = 2048;
constexpr int32_t kNoAllocMaxChunks = 32768;

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kJobsOff = 0;
constexpr size_t kChunksOff = align256(kJobsOff + sizeof(JobDesc) * kNoAllocMaxPlanes);
constexpr size_t kNoAllocScratchBytes = align256(kChunksOff + sizeof(Chunk) * kNoAllocMaxChunks);

// The scratch: the job table, then the chunk table.
static __device__ __align__(256) unsigned char g_sweep_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_sweep_scratch for the current device (looked up once).
rdct_status scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "rdct_sweep_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(RDCT_ERR_ARG, "rdct_sweep_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sweep_scratch);
        if (e != cudaSuccess || !p) return cuda_error(e, "rdct_sweep_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return RDCT_OK;
}

}  // namespace
}  // namespace rdct

using namespace rdct;

extern "C" rdct_status rdct_sweep_noalloc(const rdct_plane *planes, int32_t n, rdct_kind kind, double *sse_by_r,
                                          rdct_stream stream) {
    if (!planes || !sse_by_r || n < 0) return set_error(RDCT_ERR_ARG, "rdct_sweep_noalloc: null pointer or negative count");
    if (kind != RDCT_KIND_RDCT && kind != RDCT_KIND_DCT) return set_error(RDCT_ERR_ARG, "rdct_sweep_noalloc: bad kind");
    if (reinterpret_cast<uintptr_t>(sse_by_r) % 8) return set_error(RDCT_ERR_ARG, "rdct_sweep_noalloc: misaligned output");
    if (n > kNoAllocMaxPlanes)
        return set_error(RDCT_ERR_TOO_LARGE, "rdct_sweep_noalloc: more than 2048 planes in one call; split the call "
                                             "or use rdct_sweep");
    int64_t nchunks = 0, ntiles = 0;
    for (int32_t i = 0; i < n; ++i) {
        rdct_status st = validate_plane(&planes[i], "rdct_sweep_noalloc");
        if (st) return st;
        nchunks += sweep_chunk_count(planes[i]);
        ntiles += sweep_tiles_of(planes[i]);
    }
    if (nchunks > kNoAllocMaxChunks)
        return set_error(RDCT_ERR_TOO_LARGE, "rdct_sweep_noalloc: the planes need more than 32768 chunks of 512 "
                                             "blocks (about 1.07 Gpixel in one call); split the call or use rdct_sweep");
    if (n == 0) return RDCT_OK;
    unsigned char *base = nullptr;
    rdct_status st = scratch_address(&base);
    if (st) return st;
    JobDesc *d_jobs = reinterpret_cast<JobDesc *>(base + kJobsOff);
    Chunk *d_chunks = reinterpret_cast<Chunk *>(base + kChunksOff);
    cudaStream_t s = (cudaStream_t)stream;
    // the tables are rewritten in full by every call (from plane descriptors
    // passed as kernel parameters), and the same kernel clears the output bins
    RDCT_CUDA_TRY(build_sweep_tables(planes, n, sweep_is_tiled((int)kind), d_jobs, d_chunks, sse_by_r, s));
    RDCT_CUDA_TRY(launch_sweep(d_jobs, d_chunks, (int32_t)nchunks, (int)kind, sse_by_r, n, (int32_t)ntiles, s));
    RDCT_CUDA_TRY(launch_sweep_finalize(sse_by_r, n, (int)kind, s));
    return RDCT_OK;
}
