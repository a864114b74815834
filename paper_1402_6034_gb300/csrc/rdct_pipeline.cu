// rdct_pipeline.cu -- planes that live in host memory, streamed through the
// fused path with copies and kernels overlapped.
//
// Direct mode: the fused kernels load and store the planes in host memory
// themselves, over the host link, and nothing is staged.  It takes pinned
// planes, and also plain (pageable) host memory on a device that reaches it
// through the host's page tables (address translation over a coherent
// host-device link, as on Grace-Blackwell nodes).  Staged mode (any host memory):
// planes are cut into horizontal bands (whole block rows; 8x8 blocks are
// independent, Sec. 3), bands are packed into groups that fit one staging
// slot, and each group goes host->device on one stream, through one batch
// launch on a second, and device->host on a third.  `depth` slots rotate so
// that the copies of group g+1 and g-1 overlap the kernel of group g.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rdct_device.cuh"
#include "rdct_internal.h"

using namespace rdct;

namespace {

struct Band {
    int32_t job, row0, rows;  // rows in pixels (multiple of 8)
    int64_t off;              // byte offset of the band in the slot's input/output area
};

struct Slot {
    uint8_t *d_in = nullptr, *d_out = nullptr;
    JobDesc *d_jobs = nullptr;
    Chunk *d_chunks = nullptr;
    JobDesc *h_jobs = nullptr;  // pinned staging for the tables
    Chunk *h_chunks = nullptr;
    int32_t max_jobs = 0, max_chunks = 0;
    cudaEvent_t in_ready = nullptr, computed = nullptr, out_done = nullptr;
    bool used = false;
};

constexpr int kItemsPerChunk = 8;

}  // namespace

struct rdct_pipeline {
    int device = 0;
    int mode = RDCT_PIPELINE_AUTO;
    bool pageable_direct = false;  // the device addresses pageable host memory through the host page tables
    int64_t slot_bytes = 0;  // per direction
    std::vector<Slot> slots;
    cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
    unsigned long long *d_acc = nullptr;  // [2 * acc_cap]: 576 * SSE per image, then the 8-bit errors
    int32_t acc_cap = 0;
};

static void pipeline_free(rdct_pipeline *p) {
    if (!p) return;
    if (p->comp) cudaStreamSynchronize(p->comp);
    if (p->h2d) cudaStreamSynchronize(p->h2d);
    if (p->d2h) cudaStreamSynchronize(p->d2h);
    for (Slot &s : p->slots) {
        cudaFree(s.d_in);
        cudaFree(s.d_out);
        cudaFree(s.d_jobs);
        cudaFree(s.d_chunks);
        cudaFreeHost(s.h_jobs);
        cudaFreeHost(s.h_chunks);
        if (s.in_ready) cudaEventDestroy(s.in_ready);
        if (s.computed) cudaEventDestroy(s.computed);
        if (s.out_done) cudaEventDestroy(s.out_done);
    }
    if (p->d_acc) cudaFree(p->d_acc);
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->comp) cudaStreamDestroy(p->comp);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    delete p;
}

static rdct_status ensure_tables(Slot &s, int32_t njobs, int32_t nchunks) {
    if (njobs > s.max_jobs) {
        cudaFree(s.d_jobs);
        cudaFreeHost(s.h_jobs);
        s.d_jobs = nullptr;
        s.h_jobs = nullptr;
        const int32_t cap = std::max(njobs, 2 * s.max_jobs);
        if (cudaMalloc(&s.d_jobs, cap * sizeof(JobDesc)) != cudaSuccess ||
            cudaMallocHost(&s.h_jobs, cap * sizeof(JobDesc)) != cudaSuccess)
            return set_error(RDCT_ERR_OOM, "rdct_pipeline: table allocation failed");
        s.max_jobs = cap;
    }
    if (nchunks > s.max_chunks) {
        cudaFree(s.d_chunks);
        cudaFreeHost(s.h_chunks);
        s.d_chunks = nullptr;
        s.h_chunks = nullptr;
        const int32_t cap = std::max(nchunks, 2 * s.max_chunks);
        if (cudaMalloc(&s.d_chunks, cap * sizeof(Chunk)) != cudaSuccess ||
            cudaMallocHost(&s.h_chunks, cap * sizeof(Chunk)) != cudaSuccess)
            return set_error(RDCT_ERR_OOM, "rdct_pipeline: table allocation failed");
        s.max_chunks = cap;
    }
    return RDCT_OK;
}

// True when the device can address [p, p + bytes) with the same pointer:
// pinned (page-locked) host memory under unified addressing, or, when
// pageable_ok (the device reads and writes pageable memory through the host
// page tables), plain host memory that CUDA does not know.  The first and the
// last byte are checked; a plane is one user buffer, so both ends of one kind
// mean the buffer is of that kind as a whole.
static bool device_addressable(const void *p, int64_t bytes, bool pageable_ok) {
    const void *ends[2] = {p, static_cast<const uint8_t *>(p) + (bytes > 0 ? bytes - 1 : 0)};
    for (const void *q : ends) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        const bool pinned = a.type == cudaMemoryTypeHost && a.devicePointer == q;
        const bool pageable = pageable_ok && a.type == cudaMemoryTypeUnregistered;
        if (!pinned && !pageable) return false;
    }
    return true;
}

// Direct mode: the fused kernels read the planes from host memory and write
// the reconstructions back to host memory over the host link, with no
// staging copies; only the job and chunk tables and the per-image errors
// cross the link as copies.
static rdct_status run_direct(rdct_pipeline *p, const rdct_host_job *jobs, int32_t njobs,
                              unsigned long long *acc8) {
    std::vector<JobDesc> jd;
    std::vector<Chunk> cd;
    jd.reserve(njobs);
    for (int32_t i = 0; i < njobs; ++i) {
        const rdct_host_job &j = jobs[i];
        rdct_plane pl{j.src, j.pitch, j.w, j.h};
        JobDesc d = make_job(pl, j.dst, j.pitch, nullptr, 0, j.r, j.image, 1);
        const int items = strips_of(d, kFusedVRows);
        const int cls = fused_class_of(j.r, 2);
        for (int it = 0; it < items; it += kItemsPerChunk)
            cd.push_back(Chunk{i, it, std::min(kItemsPerChunk, items - it), cls});
        jd.push_back(d);
    }
    std::stable_sort(cd.begin(), cd.end(), [](const Chunk &a, const Chunk &b) { return a.cls < b.cls; });
    Slot &s = p->slots[0];
    rdct_status st = ensure_tables(s, (int32_t)jd.size(), (int32_t)cd.size());
    if (st) return st;
    std::memcpy(s.h_jobs, jd.data(), jd.size() * sizeof(JobDesc));
    std::memcpy(s.h_chunks, cd.data(), cd.size() * sizeof(Chunk));
    RDCT_CUDA_TRY(cudaMemcpyAsync(s.d_jobs, s.h_jobs, jd.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, p->comp));
    RDCT_CUDA_TRY(cudaMemcpyAsync(s.d_chunks, s.h_chunks, cd.size() * sizeof(Chunk), cudaMemcpyHostToDevice, p->comp));
    int32_t begin = 0;
    for (int c = 0; c < kBatchGroups; ++c) {
        int32_t end = begin;
        while (end < (int32_t)cd.size() && cd[end].cls == c) ++end;
        if (end > begin) {
            RDCT_CUDA_TRY(launch_fused_batch(s.d_jobs, s.d_chunks + begin, end - begin, p->d_acc, acc8, c, 0, 4, 2,
                                             begin > 0, p->comp));
        }
        begin = end;
    }
    return RDCT_OK;
}

// Wait for the run and hand the per-image errors to the host.
static rdct_status finish_run(rdct_pipeline *p, int32_t nimages, double *sse_per_image, double *sse_u8) {
    RDCT_CUDA_TRY(cudaStreamSynchronize(p->comp));
    RDCT_CUDA_TRY(cudaStreamSynchronize(p->d2h));
    if (nimages > 0) {
        std::vector<unsigned long long> acc(2 * (size_t)nimages);
        RDCT_CUDA_TRY(cudaMemcpy(acc.data(), p->d_acc, (size_t)nimages * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost));
        if (sse_u8)
            RDCT_CUDA_TRY(cudaMemcpy(acc.data() + nimages, p->d_acc + p->acc_cap,
                                     (size_t)nimages * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < nimages; ++i) {
            sse_per_image[i] = (double)acc[i] / 576.0;
            if (sse_u8) sse_u8[i] = (double)acc[nimages + i];
        }
    }
    return RDCT_OK;
}

extern "C" {

rdct_status rdct_pipeline_set_mode(rdct_pipeline *p, int32_t mode) {
    if (!p) return set_error(RDCT_ERR_ARG, "rdct_pipeline_set_mode: null pipeline");
    if (mode != RDCT_PIPELINE_AUTO && mode != RDCT_PIPELINE_STAGED && mode != RDCT_PIPELINE_DIRECT)
        return set_error(RDCT_ERR_ARG, "rdct_pipeline_set_mode: unknown mode");
    p->mode = mode;
    return RDCT_OK;
}

rdct_status rdct_pipeline_create(int64_t device_budget_bytes, int32_t depth, rdct_pipeline **pipe) {
    if (!pipe) return set_error(RDCT_ERR_ARG, "rdct_pipeline_create: null result");
    *pipe = nullptr;
    if (depth < 2 || depth > 16) return set_error(RDCT_ERR_ARG, "rdct_pipeline_create: depth must be in 2..16");
    if (device_budget_bytes < (int64_t)depth * 2 * (1 << 20))
        return set_error(RDCT_ERR_ARG, "rdct_pipeline_create: budget below 2 MiB per slot");
    rdct_pipeline *p = new (std::nothrow) rdct_pipeline();
    if (!p) return set_error(RDCT_ERR_OOM, "rdct_pipeline_create: host allocation failed");
    cudaGetDevice(&p->device);
    {
        int pma = 0, host_tables = 0;
        cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, p->device);
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, p->device);
        p->pageable_direct = pma == 1 && host_tables == 1;
    }
    p->slot_bytes = (device_budget_bytes / depth / 2) & ~(int64_t)255;
    p->slots.resize(depth);
    cudaError_t e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
    for (Slot &s : p->slots) {
        if (e != cudaSuccess) break;
        e = cudaMalloc(&s.d_in, p->slot_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_out, p->slot_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.in_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.computed, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        pipeline_free(p);
        return set_error(e == cudaErrorMemoryAllocation ? RDCT_ERR_OOM : RDCT_ERR_CUDA,
                         std::string("rdct_pipeline_create: ") + cudaGetErrorString(e));
    }
    *pipe = p;
    return RDCT_OK;
}

rdct_status rdct_pipeline_run(rdct_pipeline *p, const rdct_host_job *jobs, int32_t njobs, int32_t nimages,
                              double *sse_per_image, double *sse_u8_per_image) {
    if (!p || (!jobs && njobs > 0) || njobs < 0 || nimages < 0 || (!sse_per_image && nimages > 0))
        return set_error(RDCT_ERR_ARG, "rdct_pipeline_run: null or negative argument");
    for (int32_t i = 0; i < njobs; ++i) {
        const rdct_host_job &j = jobs[i];
        rdct_plane pl{j.src, j.pitch, j.w, j.h};
        rdct_status st = validate_plane(&pl, "rdct_pipeline_run");
        if (st) return st;
        if (j.r < 1 || j.r > 64) return set_error(RDCT_ERR_ARG, "rdct_pipeline_run: r must be in 1..64");
        if (j.image < 0 || j.image >= nimages) return set_error(RDCT_ERR_ARG, "rdct_pipeline_run: image out of range");
        if ((int64_t)j.w * 8 > p->slot_bytes)
            return set_error(RDCT_ERR_TOO_LARGE, "rdct_pipeline_run: a block row exceeds the staging slot");
    }
    if (nimages > p->acc_cap) {
        cudaFree(p->d_acc);
        p->d_acc = nullptr;
        p->acc_cap = 0;
        if (cudaMalloc(&p->d_acc, 2 * (size_t)nimages * sizeof(unsigned long long)) != cudaSuccess)
            return set_error(RDCT_ERR_OOM, "rdct_pipeline_run: accumulator allocation failed");
        p->acc_cap = nimages;
    }
    if (nimages > 0)
        RDCT_CUDA_TRY(cudaMemsetAsync(p->d_acc, 0, 2 * (size_t)p->acc_cap * sizeof(unsigned long long), p->comp));
    unsigned long long *acc8 = sse_u8_per_image ? p->d_acc + p->acc_cap : nullptr;

    bool direct = p->mode != RDCT_PIPELINE_STAGED;
    for (int32_t i = 0; i < njobs && direct; ++i) {
        const rdct_host_job &j = jobs[i];
        const int64_t bytes = (int64_t)(j.h - 1) * j.pitch + j.w;
        direct = device_addressable(j.src, bytes, p->pageable_direct) &&
                 (!j.dst || device_addressable(j.dst, bytes, p->pageable_direct));
    }
    if (p->mode == RDCT_PIPELINE_DIRECT && !direct)
        return set_error(RDCT_ERR_ARG, p->pageable_direct
                                           ? "rdct_pipeline_run: direct mode needs host planes (pinned or pageable)"
                                           : "rdct_pipeline_run: direct mode needs pinned host planes (this device "
                                             "does not address pageable memory)");
    if (direct) {
        rdct_status st = run_direct(p, jobs, njobs, acc8);
        if (st) return st;
        return finish_run(p, nimages, sse_per_image, sse_u8_per_image);
    }

    // cut planes into bands that fit a slot, packed 256-byte aligned, tight pitch = w
    std::vector<std::vector<Band>> groups(1);
    int64_t used = 0;
    for (int32_t i = 0; i < njobs; ++i) {
        const rdct_host_job &j = jobs[i];
        int32_t row = 0;
        while (row < j.h) {
            const int64_t room = p->slot_bytes - used;
            int64_t rows_fit = (room / j.w) & ~(int64_t)7;
            if (rows_fit <= 0) {
                groups.emplace_back();
                used = 0;
                continue;
            }
            const int32_t rows = (int32_t)std::min<int64_t>(rows_fit, j.h - row);
            groups.back().push_back(Band{i, row, rows, used});
            used += ((int64_t)rows * j.w + 255) & ~(int64_t)255;
            row += rows;
        }
    }

    int gi = 0;
    for (const std::vector<Band> &g : groups) {
        if (g.empty()) continue;
        Slot &s = p->slots[gi % p->slots.size()];
        ++gi;
        // the slot's previous group must have left the device before reuse
        if (s.used) {
            RDCT_CUDA_TRY(cudaStreamWaitEvent(p->h2d, s.out_done, 0));
            RDCT_CUDA_TRY(cudaEventSynchronize(s.computed));  // host tables of the slot are free again
        }
        // tables for this group (jobs: one per band; chunks over the bands' strips)
        std::vector<JobDesc> jd;
        std::vector<Chunk> cd;
        for (const Band &b : g) {
            const rdct_host_job &j = jobs[b.job];
            rdct_plane pl{s.d_in + b.off, j.w, j.w, b.rows};
            JobDesc d = make_job(pl, j.dst ? s.d_out + b.off : nullptr, j.w, nullptr, 0, j.r, j.image, 1);
            const int items = strips_of(d, kFusedVRows);
            const int cls = fused_class_of(j.r, 2);
            for (int it = 0; it < items; it += kItemsPerChunk)
                cd.push_back(Chunk{(int32_t)jd.size(), it, std::min(kItemsPerChunk, items - it), cls});
            jd.push_back(d);
        }
        std::stable_sort(cd.begin(), cd.end(), [](const Chunk &a, const Chunk &b) { return a.cls < b.cls; });
        rdct_status st = ensure_tables(s, (int32_t)jd.size(), (int32_t)cd.size());
        if (st) return st;
        std::memcpy(s.h_jobs, jd.data(), jd.size() * sizeof(JobDesc));
        std::memcpy(s.h_chunks, cd.data(), cd.size() * sizeof(Chunk));
        for (const Band &b : g) {
            const rdct_host_job &j = jobs[b.job];
            RDCT_CUDA_TRY(cudaMemcpy2DAsync(s.d_in + b.off, j.w, j.src + (int64_t)b.row0 * j.pitch, j.pitch, j.w,
                                            b.rows, cudaMemcpyHostToDevice, p->h2d));
        }
        RDCT_CUDA_TRY(cudaMemcpyAsync(s.d_jobs, s.h_jobs, jd.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, p->h2d));
        RDCT_CUDA_TRY(cudaMemcpyAsync(s.d_chunks, s.h_chunks, cd.size() * sizeof(Chunk), cudaMemcpyHostToDevice, p->h2d));
        RDCT_CUDA_TRY(cudaEventRecord(s.in_ready, p->h2d));
        RDCT_CUDA_TRY(cudaStreamWaitEvent(p->comp, s.in_ready, 0));
        int32_t begin = 0;
        for (int c = 0; c < kBatchGroups; ++c) {
            int32_t end = begin;
            while (end < (int32_t)cd.size() && cd[end].cls == c) ++end;
            if (end > begin) {
                RDCT_CUDA_TRY(launch_fused_batch(s.d_jobs, s.d_chunks + begin, end - begin, p->d_acc, acc8, c, 0, 4,
                                                 2, begin > 0, p->comp));
            }
            begin = end;
        }
        RDCT_CUDA_TRY(cudaEventRecord(s.computed, p->comp));
        RDCT_CUDA_TRY(cudaStreamWaitEvent(p->d2h, s.computed, 0));
        for (const Band &b : g) {
            const rdct_host_job &j = jobs[b.job];
            if (!j.dst) continue;
            RDCT_CUDA_TRY(cudaMemcpy2DAsync(j.dst + (int64_t)b.row0 * j.pitch, j.pitch, s.d_out + b.off, j.w, j.w,
                                            b.rows, cudaMemcpyDeviceToHost, p->d2h));
        }
        RDCT_CUDA_TRY(cudaEventRecord(s.out_done, p->d2h));
        s.used = true;
    }
    return finish_run(p, nimages, sse_per_image, sse_u8_per_image);
}

rdct_status rdct_pipeline_destroy(rdct_pipeline *p) {
    pipeline_free(p);
    return RDCT_OK;
}

}  // extern "C"
