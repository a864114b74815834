// rdct_server.cu -- a serving loop for the fused RDCT path with continuous
// batching.
//
// Requests (images of 1..3 planes in host memory, each with its own r) are
// queued by rdct_server_submit.  One scheduler thread:
//   1. admits queued requests in arrival order while their buffers fit the
//      device-memory budget (a first-fit arena with coalescing; a request that
//      does not fit waits, it is never reordered past);
//   2. copies each admitted request host->device on a copy stream as soon as
//      it is admitted, so copies overlap kernels already running;
//   3. whenever one of the compute streams is free, launches every admitted,
//      copied request (up to max_batch) as one batch: one persistent kernel
//      per r present over a flattened strip index, then the device->host
//      copies of the reconstructions and per-image errors;
//   4. polls completion events, finishes results, frees buffers and wakes
//      waiters.
// Requests that arrive while launches are in flight join the next launch
// (continuous batching); their work overlaps other batches on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#if defined(__linux__)
#include <sys/prctl.h>
#endif

#include "rdct_device.cuh"
#include "rdct_internal.h"

using namespace rdct;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kServerItemsPerChunk = 8;
// Interval at which the scheduler polls the completion events of launches in
// flight (it wakes at once for new requests).
constexpr int kPollUs = 10;

struct Req {
    uint64_t ticket = 0;
    rdct_request q{};
    int64_t bytes = 0;        // device bytes (input + output planes)
    int64_t arena_off = -1;
    Clock::time_point t_submit, t_admit;
    cudaEvent_t copied = nullptr;
    bool src_pageable = false, dst_pageable = false;  // moved by copy kernels (see rdct_server.pageable)
    bool admitted = false;
    rdct_result res{};
    bool done = false;
};

struct Lane {  // one compute stream and its per-launch resources
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    JobDesc *d_jobs = nullptr, *h_jobs = nullptr;
    Chunk *d_chunks = nullptr, *h_chunks = nullptr;
    unsigned long long *d_acc = nullptr, *h_acc = nullptr;  // per request: 576 * SSE, then the 8-bit error
    int32_t cap_jobs = 0, cap_chunks = 0, cap_acc = 0;
    std::vector<std::shared_ptr<Req>> batch;
    bool busy = false;
};

}  // namespace

struct rdct_server {
    rdct_server_opts opts{};
    int device = 0;
    uint8_t *d_pool = nullptr;
    rdct_arena *arena = nullptr;
    cudaStream_t copy = nullptr;
    std::vector<Lane> lanes;
    // the device reads and writes pageable host memory through the host page
    // tables: request planes in such memory are moved by copy kernels, which
    // stay asynchronous, instead of the copy engines (whose pageable copies
    // the driver stages, synchronously)
    bool pageable = false;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<Req>> queue;    // submitted, not admitted
    std::deque<std::shared_ptr<Req>> ready;    // admitted, copy issued, not launched
    std::map<uint64_t, std::shared_ptr<Req>> all;  // every live ticket
    uint64_t next_ticket = 1;
    bool stop = false;
    int fail_allocs = 0;  // test hook: the next n arena allocations fail
    std::thread th;

    // stats
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, alloc_failures = 0;
    int64_t peak_resident = 0;
    double samples_done = 0;
    Clock::time_point t_first{}, t_last{};
    bool any = false;
    std::vector<double> lat_us;
};

namespace {

bool request_bytes(const rdct_request &q, int64_t *bytes) {
    const int64_t plane = (int64_t)q.w * q.h;
    *bytes = 2 * plane * q.planes;
    return true;
}

rdct_status validate_request(const rdct_request *q) {
    if (!q || !q->src) return set_error(RDCT_ERR_ARG, "rdct_server_submit: null request or source");
    if (q->planes < 1 || q->planes > 4) return set_error(RDCT_ERR_ARG, "rdct_server_submit: planes must be 1..4");
    if (q->w <= 0 || q->h <= 0 || q->w % 8 || q->h % 8 || q->pitch < q->w)
        return set_error(RDCT_ERR_SHAPE, "rdct_server_submit: sides must be positive multiples of 8, pitch >= w");
    if (q->r < 1 || q->r > 64) return set_error(RDCT_ERR_ARG, "rdct_server_submit: r must be in 1..64");
    if (q->plane_stride != 0 && q->planes > 1 && q->plane_stride < q->pitch * (q->h - 1) + q->w)
        return set_error(RDCT_ERR_ARG, "rdct_server_submit: planes overlap (plane_stride too small)");
    return RDCT_OK;
}

// Grows one table pair (device + pinned host) of a lane to at least n
// elements.  Called only while the lane is idle (its last batch completed),
// so the old device table is released in stream order instead of by a
// device-wide synchronising cudaFree.  Tables are sized at server creation
// for a full budget, so this runs only for unusually fragmented batches.
template <typename T>
bool grow_table(cudaStream_t s, T *&d, T *&h, int32_t &cap, int32_t n) {
    if (n <= cap) return true;
    if (d) cudaFreeAsync(d, s);
    if (h) cudaFreeHost(h);
    d = nullptr;
    h = nullptr;
    cap = std::max(n, 2 * cap);
    if (cudaMallocAsync(reinterpret_cast<void **>(&d), (size_t)cap * sizeof(T), s) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&h), (size_t)cap * sizeof(T)) != cudaSuccess) {
        cap = 0;
        return false;
    }
    return true;
}

bool grow(Lane &L, int32_t njobs, int32_t nchunks, int32_t nacc) {
    return grow_table(L.s, L.d_jobs, L.h_jobs, L.cap_jobs, njobs) &&
           grow_table(L.s, L.d_chunks, L.h_chunks, L.cap_chunks, nchunks) &&
           grow_table(L.s, L.d_acc, L.h_acc, L.cap_acc, nacc);
}

// Chunks a batch can need when the whole budget holds its planes: a chunk
// covers kServerItemsPerChunk items of 32 column pairs, and a pair holds at
// least one 8x8 block of input (two unless it is in the last block row of a
// plane with an odd number of them); every plane adds at most one partial
// chunk.  Capped so that a very large budget does not pin a large table up
// front (larger batches still grow the table).
int32_t chunk_bound(const rdct_server_opts &o) {
    const int64_t chunk_input = (int64_t)kServerItemsPerChunk * 32 * 64;
    const int64_t n = o.device_budget_bytes / 2 / chunk_input + 8 * (int64_t)o.max_batch + 64;
    return (int32_t)std::min<int64_t>(n, 1 << 20);
}

void finish(rdct_server *S, Req &r, rdct_status st, Clock::time_point now) {
    r.res.status = st;
    r.res.latency_us = std::chrono::duration<double, std::micro>(now - r.t_submit).count();
    r.done = true;
}

// Launch one batch on lane L (caller holds no lock; L.batch already filled).
rdct_status launch_batch(rdct_server *S, Lane &L) {
    std::vector<JobDesc> jobs;
    std::vector<Chunk> chunks;
    const int32_t n = (int32_t)L.batch.size();
    for (int32_t i = 0; i < n; ++i) {
        Req &r = *L.batch[i];
        const int64_t plane = (int64_t)r.q.w * r.q.h;
        uint8_t *base = S->d_pool + r.arena_off;
        for (int p = 0; p < r.q.planes; ++p) {
            rdct_plane pl{base + p * plane, r.q.w, r.q.w, r.q.h};
            uint8_t *dst = r.q.dst ? base + (r.q.planes + p) * plane : nullptr;
            JobDesc d = make_job(pl, dst, r.q.w, nullptr, 0, r.q.r, i, 1);
            const int items = strips_of(d, kFusedVRows);
            const int cls = fused_class_of(r.q.r, 2);
            for (int it = 0; it < items; it += kServerItemsPerChunk)
                chunks.push_back(Chunk{(int32_t)jobs.size(), it, std::min(kServerItemsPerChunk, items - it), cls});
            jobs.push_back(d);
        }
        RDCT_CUDA_TRY(cudaStreamWaitEvent(L.s, r.copied, 0));
    }
    std::stable_sort(chunks.begin(), chunks.end(), [](const Chunk &a, const Chunk &b) { return a.cls < b.cls; });
    if (!grow(L, (int32_t)jobs.size(), (int32_t)chunks.size(), 2 * n))
        return set_error(RDCT_ERR_OOM, "rdct_server: table allocation failed");
    std::memcpy(L.h_jobs, jobs.data(), jobs.size() * sizeof(JobDesc));
    std::memcpy(L.h_chunks, chunks.data(), chunks.size() * sizeof(Chunk));
    RDCT_CUDA_TRY(cudaMemcpyAsync(L.d_jobs, L.h_jobs, jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, L.s));
    RDCT_CUDA_TRY(cudaMemcpyAsync(L.d_chunks, L.h_chunks, chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice, L.s));
    RDCT_CUDA_TRY(cudaMemsetAsync(L.d_acc, 0, 2 * n * sizeof(unsigned long long), L.s));
    int32_t begin = 0;
    while (begin < (int32_t)chunks.size()) {
        int32_t end = begin;
        while (end < (int32_t)chunks.size() && chunks[end].cls == chunks[begin].cls) ++end;
        RDCT_CUDA_TRY(launch_fused_batch(L.d_jobs, L.d_chunks + begin, end - begin, L.d_acc, L.d_acc + n,
                                         chunks[begin].cls, 0, 4, 2, begin > 0, L.s));
        begin = end;
    }
    for (int32_t i = 0; i < n; ++i) {
        Req &r = *L.batch[i];
        if (!r.q.dst) continue;
        const int64_t plane = (int64_t)r.q.w * r.q.h;
        uint8_t *out = S->d_pool + r.arena_off + r.q.planes * plane;
        for (int p = 0; p < r.q.planes; ++p) {
            if (r.dst_pageable)
                RDCT_CUDA_TRY(launch_copy2d(r.q.dst + p * r.q.plane_stride, r.q.pitch, out + p * plane, r.q.w, r.q.w,
                                            r.q.h, L.s));
            else
                RDCT_CUDA_TRY(cudaMemcpy2DAsync(r.q.dst + p * r.q.plane_stride, r.q.pitch, out + p * plane,
                                                r.q.w, r.q.w, r.q.h, cudaMemcpyDeviceToHost, L.s));
        }
    }
    RDCT_CUDA_TRY(cudaMemcpyAsync(L.h_acc, L.d_acc, 2 * n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, L.s));
    RDCT_CUDA_TRY(cudaEventRecord(L.done, L.s));
    return RDCT_OK;
}

void scheduler(rdct_server *S) {
    cudaSetDevice(S->device);
#if defined(PR_SET_TIMERSLACK)
    // The loop polls in-flight launches every few microseconds; with the default
    // timer slack of an ordinary thread (50 us on Linux) each short timed wait
    // could oversleep by that much and delay every completion.
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool inflight = false;
        for (Lane &L : S->lanes) inflight |= L.busy;
        if (S->stop && S->queue.empty() && S->ready.empty() && !inflight) break;
        if (S->queue.empty() && S->ready.empty() && !inflight) {
            S->cv_sched.wait(lk);
            continue;
        }
        const Clock::time_point now = Clock::now();
        // 1. completions
        bool freed = false;
        for (Lane &L : S->lanes) {
            if (!L.busy) continue;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            const rdct_status st = q == cudaSuccess ? RDCT_OK : RDCT_ERR_CUDA;
            const Clock::time_point t = Clock::now();
            const int32_t nb = (int32_t)L.batch.size();
            for (int32_t i = 0; i < nb; ++i) {
                Req &r = *L.batch[i];
                const double n = (double)r.q.w * r.q.h * r.q.planes;
                r.res.sse = st == RDCT_OK ? (double)L.h_acc[i] / 576.0 : 0.0;
                r.res.mse = r.res.sse / n;
                r.res.psnr = r.res.mse == 0.0 ? INFINITY : 10.0 * std::log10(255.0 * 255.0 / r.res.mse);
                r.res.sse_u8 = st == RDCT_OK ? (double)L.h_acc[nb + i] : 0.0;
                r.res.mse_u8 = r.res.sse_u8 / n;
                r.res.psnr_u8 = r.res.mse_u8 == 0.0 ? INFINITY : 10.0 * std::log10(255.0 * 255.0 / r.res.mse_u8);
                finish(S, r, st, t);
                rdct_arena_free(S->arena, r.arena_off);
                cudaEventDestroy(r.copied);
                r.copied = nullptr;
                S->completed++;
                S->samples_done += n;
                S->lat_us.push_back(r.res.latency_us);
                S->t_last = t;
            }
            L.batch.clear();
            L.busy = false;
            freed = true;
        }
        if (freed) S->cv_done.notify_all();
        // 2. admission in arrival order
        while (!S->queue.empty()) {
            std::shared_ptr<Req> r = S->queue.front();
            int64_t off = -1;
            if (S->fail_allocs > 0) {
                S->fail_allocs--;
                S->alloc_failures++;
                break;  // injected failure: the request stays queued and is retried
            }
            if (rdct_arena_alloc(S->arena, r->bytes, &off) != RDCT_OK) break;
            S->queue.pop_front();
            r->arena_off = off;
            r->admitted = true;
            r->t_admit = Clock::now();
            S->peak_resident = std::max(S->peak_resident, rdct_arena_used(S->arena));
            const int64_t plane = (int64_t)r->q.w * r->q.h;
            cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming);
            for (int p = 0; p < r->q.planes; ++p) {
                if (r->src_pageable)
                    launch_copy2d(S->d_pool + off + p * plane, r->q.w, r->q.src + p * r->q.plane_stride, r->q.pitch,
                                  r->q.w, r->q.h, S->copy);
                else
                    cudaMemcpy2DAsync(S->d_pool + off + p * plane, r->q.w, r->q.src + p * r->q.plane_stride,
                                      r->q.pitch, r->q.w, r->q.h, cudaMemcpyHostToDevice, S->copy);
            }
            cudaEventRecord(r->copied, S->copy);
            S->ready.push_back(r);
        }
        // 3. launches on free lanes; a partial batch waits up to max_wait_us
        //    for company while more requests are queued
        for (Lane &L : S->lanes) {
            if (L.busy || S->ready.empty()) continue;
            if ((int32_t)S->ready.size() < S->opts.max_batch && !S->queue.empty() && S->opts.max_wait_us > 0 &&
                Clock::now() - S->ready.front()->t_admit < std::chrono::microseconds(S->opts.max_wait_us))
                continue;
            while (!S->ready.empty() && (int32_t)L.batch.size() < S->opts.max_batch) {
                L.batch.push_back(S->ready.front());
                S->ready.pop_front();
            }
            // the batch's requests are admitted (not cancellable) and only this
            // thread touches the lane, so submitters need not wait for the launch
            lk.unlock();
            const rdct_status st = launch_batch(S, L);
            lk.lock();
            S->batches++;
            if (st != RDCT_OK) {
                const Clock::time_point t = Clock::now();
                for (auto &r : L.batch) {
                    finish(S, *r, st, t);
                    rdct_arena_free(S->arena, r->arena_off);
                    if (r->copied) cudaEventDestroy(r->copied);
                    r->copied = nullptr;
                }
                L.batch.clear();
                S->cv_done.notify_all();
                continue;
            }
            L.busy = true;
        }
        // 4. wait for the next event: new requests, or poll in-flight work
        bool busy = false;
        for (Lane &L : S->lanes) busy |= L.busy;
        if (busy) S->cv_sched.wait_for(lk, std::chrono::microseconds(kPollUs));
        else if (!S->ready.empty() || (!S->queue.empty() && S->fail_allocs == 0))
            S->cv_sched.wait_for(lk, std::chrono::microseconds(20));
        else if (!S->queue.empty())
            S->cv_sched.wait_for(lk, std::chrono::microseconds(200));
        (void)now;
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double idx = p * (v.size() - 1);
    const size_t lo = (size_t)idx, hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (idx - lo);
}

void server_free(rdct_server *S) {
    for (Lane &L : S->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        if (L.d_jobs) cudaFree(L.d_jobs);
        cudaFreeHost(L.h_jobs);
        if (L.d_chunks) cudaFree(L.d_chunks);
        cudaFreeHost(L.h_chunks);
        if (L.d_acc) cudaFree(L.d_acc);
        cudaFreeHost(L.h_acc);
        if (L.done) cudaEventDestroy(L.done);
        if (L.s) cudaStreamDestroy(L.s);
    }
    if (S->copy) {
        cudaStreamSynchronize(S->copy);
        cudaStreamDestroy(S->copy);
    }
    if (S->d_pool) cudaFree(S->d_pool);
    if (S->arena) rdct_arena_destroy(S->arena);
    delete S;
}

}  // namespace

extern "C" {

rdct_status rdct_server_create(const rdct_server_opts *opts, rdct_server **server) {
    if (!opts || !server) return set_error(RDCT_ERR_ARG, "rdct_server_create: null argument");
    *server = nullptr;
    if (opts->device_budget_bytes < (1 << 20) || opts->max_batch < 1 || opts->queue_capacity < 1 || opts->streams < 1 ||
        opts->streams > 16 || opts->max_wait_us < 0)
        return set_error(RDCT_ERR_ARG, "rdct_server_create: budget >= 1 MiB, max_batch >= 1, queue_capacity >= 1, "
                                       "streams 1..16, max_wait_us >= 0");
    rdct_server *S = new (std::nothrow) rdct_server();
    if (!S) return set_error(RDCT_ERR_OOM, "rdct_server_create: host allocation failed");
    S->opts = *opts;
    cudaGetDevice(&S->device);
    S->pageable = device_pageable_access(S->device);
    if (cudaMalloc(&S->d_pool, opts->device_budget_bytes) != cudaSuccess) {
        server_free(S);
        return set_error(RDCT_ERR_OOM, "rdct_server_create: device budget allocation failed");
    }
    rdct_status st = rdct_arena_create(opts->device_budget_bytes, 256, &S->arena);
    if (st) {
        server_free(S);
        return st;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking);
    S->lanes.resize(opts->streams);
    for (Lane &L : S->lanes) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e == cudaSuccess && !grow(L, 4 * opts->max_batch, chunk_bound(*opts), 2 * opts->max_batch))
            e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        server_free(S);
        return cuda_error(e, "rdct_server_create");
    }
    S->th = std::thread(scheduler, S);
    *server = S;
    return RDCT_OK;
}

rdct_status rdct_server_submit(rdct_server *S, const rdct_request *req, uint64_t *ticket) {
    if (!S || !ticket) return set_error(RDCT_ERR_ARG, "rdct_server_submit: null argument");
    rdct_status st = validate_request(req);
    if (st) return st;
    auto r = std::make_shared<Req>();
    r->q = *req;
    if (r->q.plane_stride == 0) r->q.plane_stride = r->q.pitch * r->q.h;
    request_bytes(*req, &r->bytes);
    r->bytes = (r->bytes + 255) & ~(int64_t)255;
    if (S->pageable) {
        const int64_t extent = (int64_t)(r->q.planes - 1) * r->q.plane_stride + (int64_t)(r->q.h - 1) * r->q.pitch + r->q.w;
        r->src_pageable = is_pageable_host(r->q.src, extent);
        r->dst_pageable = r->q.dst && is_pageable_host(r->q.dst, extent);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return set_error(RDCT_ERR_BUSY, "rdct_server_submit: server is shutting down");
    if (r->bytes > S->opts.device_budget_bytes) {
        S->rejected++;
        return set_error(RDCT_ERR_TOO_LARGE, "rdct_server_submit: request larger than the device budget");
    }
    if ((int32_t)S->queue.size() >= S->opts.queue_capacity) {
        S->rejected++;
        return set_error(RDCT_ERR_BUSY, "rdct_server_submit: queue full");
    }
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    if (!S->any) {
        S->any = true;
        S->t_first = r->t_submit;
    }
    S->queue.push_back(r);
    S->all[r->ticket] = r;
    S->submitted++;
    *ticket = r->ticket;
    S->cv_sched.notify_one();
    return RDCT_OK;
}

rdct_status rdct_server_wait(rdct_server *S, uint64_t ticket, int64_t timeout_us, rdct_result *result) {
    if (!S) return set_error(RDCT_ERR_ARG, "rdct_server_wait: null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return set_error(RDCT_ERR_NOT_FOUND, "rdct_server_wait: unknown ticket");
    std::shared_ptr<Req> r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_us < 0) S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
        return set_error(RDCT_ERR_TIMEOUT, "rdct_server_wait: timed out");
    if (result) *result = r->res;
    S->all.erase(ticket);
    return r->res.status == RDCT_OK ? RDCT_OK : set_error(r->res.status, "rdct_server_wait: request failed");
}

rdct_status rdct_server_poll(rdct_server *S, uint64_t ticket, rdct_result *result) {
    if (!S) return set_error(RDCT_ERR_ARG, "rdct_server_poll: null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return set_error(RDCT_ERR_NOT_FOUND, "rdct_server_poll: unknown ticket");
    if (!it->second->done) return RDCT_ERR_BUSY;
    if (result) *result = it->second->res;
    const rdct_status st = it->second->res.status;
    S->all.erase(it);
    return st;
}

rdct_status rdct_server_cancel(rdct_server *S, uint64_t ticket) {
    if (!S) return set_error(RDCT_ERR_ARG, "rdct_server_cancel: null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return set_error(RDCT_ERR_NOT_FOUND, "rdct_server_cancel: unknown ticket");
    std::shared_ptr<Req> r = it->second;
    if (r->admitted || r->done) return set_error(RDCT_ERR_BUSY, "rdct_server_cancel: already admitted");
    S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), r), S->queue.end());
    finish(S, *r, RDCT_ERR_CANCELLED, Clock::now());
    S->cv_done.notify_all();
    return RDCT_OK;
}

rdct_status rdct_server_stats_get(rdct_server *S, rdct_server_stats *st) {
    if (!S || !st) return set_error(RDCT_ERR_ARG, "rdct_server_stats_get: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->batches = S->batches;
    st->p50_us = percentile(S->lat_us, 0.50);
    st->p99_us = percentile(S->lat_us, 0.99);
    st->p999_us = percentile(S->lat_us, 0.999);
    double sum = 0;
    for (double v : S->lat_us) sum += v;
    st->mean_us = S->lat_us.empty() ? 0.0 : sum / S->lat_us.size();
    const double secs = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    st->gpixels_per_s = secs > 0 ? S->samples_done / secs / 1e9 : 0.0;
    st->peak_resident_bytes = S->peak_resident;
    return RDCT_OK;
}

rdct_status rdct_server_destroy(rdct_server *S) {
    if (!S) return RDCT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->fail_allocs = 0;
    }
    S->cv_sched.notify_all();
    if (S->th.joinable()) S->th.join();
    server_free(S);
    return RDCT_OK;
}

rdct_status rdct_server_inject_alloc_failures(rdct_server *S, int32_t n) {
    if (!S || n < 0) return set_error(RDCT_ERR_ARG, "rdct_server_inject_alloc_failures: bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    S->fail_allocs = n;
    S->cv_sched.notify_one();
    return RDCT_OK;
}

}  // extern "C"
