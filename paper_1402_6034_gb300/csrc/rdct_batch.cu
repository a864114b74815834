// rdct_batch.cu -- batches of uneven planes in one graph launch, and the
// autotuner that picks the launch shape.
//
// The paper runs its experiment image by image (Sec. 3).  Here every plane of
// a batch is cut into work items (32 column pairs of two 8x8 blocks for the
// per-thread-copy kernel, a 32-column segment of a row pair for the TMA-staged
// one; one block row of 32 blocks for the scalar kernel), items are grouped
// into chunks, and the chunk table is walked by persistent warps, so a batch
// of thousands of planes of different sizes and r costs one graph launch.
// The retained-coefficient count r varies per plane; chunks are ordered by r
// (and staging form) and each group gets its own specialised kernel launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "rdct_device.cuh"
#include "rdct_fused2.cuh"
#include "rdct_internal.h"

using namespace rdct;

struct rdct_plan {
    int device = 0;
    int32_t nimages = 0;
    rdct_tune tune{};
    std::vector<JobDesc> jobs;     // host copy, segs computed for the plan's tile
    std::vector<JobDesc> jobs_pp;  // per-plane launches (one block per thread)
    std::vector<Chunk> chunks;
    // chunk ranges per launch group: groups 0..kBatchGroups-1 per-thread
    // copies, kBatchGroups.. the same classes with TMA staging
    int32_t group_begin[2 * kBatchGroups + 1] = {0};
    JobDesc *d_jobs = nullptr;
    Chunk *d_chunks = nullptr;
    bool tma = false;                // some jobs use the TMA-staged kernel (items: row pair x 32-column segment)
    bool balance_chunks = false;     // default tune: chunk sizes chosen per r so that the warps get equal shares
    std::vector<unsigned char> maps; // two encoded tensor maps per job (zeros for jobs without TMA)
    std::vector<char> job_tma;       // per job: TMA staging
    unsigned char *d_maps = nullptr;
    // graph cache: one executable for the last (sse, sse_u8) pointers
    std::mutex mu;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *exec_sse = nullptr, *exec_sse8 = nullptr;
};

namespace {

// TMA staging (one box request per warp and item instead of sixteen copies
// per thread) pays where the kernel is bound by instruction issue: r from 16
// (anti-diagonal 5) up.  Below, where the kernel runs at the copy bandwidth,
// the per-thread copies measured faster (their items run on across row ends,
// so no lane idles at a plane's right edge).
// A TMA item is a 32-column segment of a row pair, so a plane whose width in
// blocks is not a multiple of 32 leaves lanes of its last segment idle, where
// the per-thread copies run on into the next row.  Measured on 4096 uneven
// planes: TMA only where at most 1/16 of the segment lanes idle (+1%).
bool tma_pays(int r) { return diag_class_host(r) >= 5; }
bool tma_pays_plane(const JobDesc &j) {
    const int segw = 32 * ((j.nbw + 31) / 32);
    return tma_pays(j.r) && 16 * (segw - j.nbw) <= segw;
}

rdct_tune default_tune() {
    rdct_tune t{};
    t.warps_per_cta = 4;
    t.ctas_per_sm = 0;  // occupancy limit
    t.items_per_chunk = 16;
    t.blocks_per_thread = 2;
    t.staging = 0;
    return t;
}

rdct_status validate_tune(const rdct_tune &t) {
    if (t.warps_per_cta < 1 || t.warps_per_cta > 8 || t.ctas_per_sm < 0 || t.ctas_per_sm > 64 ||
        t.items_per_chunk < 1 || t.items_per_chunk > 4096 || (t.blocks_per_thread != 1 && t.blocks_per_thread != 2) ||
        (t.staging != 0 && t.staging != 1))
        return set_error(RDCT_ERR_ARG, "rdct_tune: out of range (warps 1..8, ctas_per_sm 0..64, "
                                       "items_per_chunk 1..4096, blocks_per_thread 1 or 2, staging 0 or 1)");
    return RDCT_OK;
}

bool same_tune(const rdct_tune &a, const rdct_tune &b) {
    return a.warps_per_cta == b.warps_per_cta && a.ctas_per_sm == b.ctas_per_sm &&
           a.items_per_chunk == b.items_per_chunk && a.blocks_per_thread == b.blocks_per_thread &&
           a.staging == b.staging;
}

rdct_status validate_jobs(const rdct_job *jobs, int32_t njobs, int32_t nimages) {
    if (!jobs && njobs > 0) return set_error(RDCT_ERR_ARG, "batch: null job array");
    if (njobs < 0 || nimages < 0) return set_error(RDCT_ERR_ARG, "batch: negative count");
    for (int32_t i = 0; i < njobs; ++i) {
        const rdct_job &j = jobs[i];
        const std::string what = "batch job " + std::to_string(i);
        rdct_status st = validate_plane(&j.src, what.c_str());
        if (st) return st;
        if (j.r < 1 || j.r > 64) return set_error(RDCT_ERR_ARG, "job " + std::to_string(i) + ": r must be in 1..64");
        if (j.image < 0 || j.image >= nimages)
            return set_error(RDCT_ERR_ARG, "job " + std::to_string(i) + ": image index out of range");
        if (j.dst && j.dst_pitch < j.src.w)
            return set_error(RDCT_ERR_SHAPE, "job " + std::to_string(i) + ": dst pitch smaller than width");
    }
    return RDCT_OK;
}

// CTAs per SM of the two-block kernel for r (its launch bounds, at most kFused2MaxCtas).
template <int... I>
constexpr int fused2_min_blocks(int r, std::integer_sequence<int, I...>) {
    int v = kFused2MaxCtas;
    ((v = (r == I + 1) ? Fused2Shape<I + 1>::min_blocks : v), ...);
    return v;
}
int fused2_ctas_per_sm(int r) {
    const int m = fused2_min_blocks(r, std::make_integer_sequence<int, 64>{});
    return m < kFused2MaxCtas ? m : kFused2MaxCtas;
}

// Items per chunk for one persistent two-block launch of `items` work items
// over `nwarps` warps, which take chunks c = warp, warp + nwarps, ...: the
// largest size up to `per` whose rounds leave the warps at least 97 % evenly
// loaded (the most even one if none does).  A small batch thus gets smaller
// chunks; a large one keeps `per`.
int balanced_chunk(int64_t items, int64_t nwarps, int per) {
    if (items <= 0 || nwarps <= 0) return per;
    int best = per;
    double best_eff = 0.0;
    for (int c = per; c >= 1; --c) {
        const int64_t chunks = (items + c - 1) / c;
        const int64_t rounds = (chunks + nwarps - 1) / nwarps;
        const double eff = (double)items / ((double)nwarps * (double)c * (double)rounds);
        if (eff >= 0.97) return c;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = c;
        }
    }
    return best;
}

void build_tables(rdct_plan *p, const rdct_job *jobs, int32_t njobs) {
    const int vrows = p->tune.blocks_per_thread == 2 ? kFusedVRows : 1;
    p->jobs.resize(njobs);
    p->jobs_pp.resize(njobs);
    for (int32_t i = 0; i < njobs; ++i) {
        const rdct_job &j = jobs[i];
        p->jobs[i] = make_job(j.src, j.dst, j.dst_pitch, nullptr, 0, j.r, j.image, 1);
        p->jobs_pp[i] = p->jobs[i];
    }
    // TMA staging per job: two blocks per thread, an r where it pays, and a
    // plane (and reconstruction) whose tensor maps encode
    const bool tma_ok = p->tune.blocks_per_thread == 2 && p->tune.staging == 0 && njobs > 0 && tma_available();
    p->job_tma.assign(njobs, 0);
    p->maps.clear();
    p->tma = false;
    if (tma_ok) {
        p->maps.assign((size_t)njobs * 2 * kTensorMapBytes, 0);
        for (int32_t i = 0; i < njobs; ++i) {
            if (!tma_pays_plane(p->jobs[i])) continue;
            p->job_tma[i] = tma_encode_plane(p->jobs[i], p->maps.data() + (size_t)i * 2 * kTensorMapBytes) ? 1 : 0;
            p->tma = p->tma || p->job_tma[i];
        }
        if (!p->tma) p->maps.clear();
    }
    std::vector<Chunk> ch;
    const int per = p->tune.items_per_chunk;
    // chunk size per launch class (one persistent launch per class and staging form)
    std::vector<int> per_class(2 * kBatchGroups, per);
    if (p->balance_chunks && p->tune.blocks_per_thread == 2) {
        std::vector<int64_t> items_of_class(2 * kBatchGroups, 0);
        for (int32_t i = 0; i < njobs; ++i) {
            const bool t = p->job_tma[i] != 0;
            items_of_class[fused_class_of(p->jobs[i].r, 2) + (t ? kBatchGroups : 0)] +=
                t ? tma_items_of(p->jobs[i]) : strips_of(p->jobs[i], vrows);
        }
        for (int c = 0; c < 2 * kBatchGroups; ++c) {
            if (!items_of_class[c]) continue;
            const int r = (c % kBatchGroups) + 1;  // two-block classes are r - 1
            int ctas = fused2_ctas_per_sm(r);
            if (p->tune.ctas_per_sm > 0 && p->tune.ctas_per_sm < ctas) ctas = p->tune.ctas_per_sm;
            per_class[c] = balanced_chunk(items_of_class[c], (int64_t)sm_count() * ctas * 4, per);
        }
    }
    for (int32_t i = 0; i < njobs; ++i) {
        const bool t = p->job_tma[i] != 0;
        const int items = t ? tma_items_of(p->jobs[i]) : strips_of(p->jobs[i], vrows);
        const int c = fused_class_of(p->jobs[i].r, p->tune.blocks_per_thread) + (t ? kBatchGroups : 0);
        const int pc = per_class[c];
        for (int it = 0; it < items; it += pc) ch.push_back(Chunk{i, it, std::min(pc, items - it), c});
    }
    std::stable_sort(ch.begin(), ch.end(), [](const Chunk &a, const Chunk &b) { return a.cls < b.cls; });
    p->chunks = std::move(ch);
    const int bpt = p->tune.blocks_per_thread;
    for (int g = 0; g <= 2 * kBatchGroups; ++g) p->group_begin[g] = 0;
    for (const Chunk &c : p->chunks) {
        const bool t = c.cls >= kBatchGroups;
        p->group_begin[batch_group_of_class(c.cls - (t ? kBatchGroups : 0), bpt) + (t ? kBatchGroups : 0) + 1]++;
    }
    for (int g = 0; g < 2 * kBatchGroups; ++g) p->group_begin[g + 1] += p->group_begin[g];
}

// memset -> one persistent kernel per non-empty group, in stream order (the
// groups overlap only at their tails; running them as parallel graph branches
// measured slower) -> in-place 576*SSE to SSE (and the 8-bit errors to double).
cudaError_t enqueue_batch(rdct_plan *p, double *sse, double *sse8, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sse, 0, (size_t)p->nimages * sizeof(double), s);
    if (e == cudaSuccess && sse8) e = cudaMemsetAsync(sse8, 0, (size_t)p->nimages * sizeof(double), s);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(sse);
    unsigned long long *acc8 = reinterpret_cast<unsigned long long *>(sse8);
    bool first = true;
    for (int g = 0; g < 2 * kBatchGroups && e == cudaSuccess; ++g) {
        const int32_t b = p->group_begin[g], n = p->group_begin[g + 1] - b;
        if (n == 0) continue;
        if (g >= kBatchGroups)
            e = launch_fused2_tma_batch(p->d_jobs, p->d_chunks + b, n, p->d_maps, acc, acc8, g - kBatchGroups + 1,
                                        p->tune.ctas_per_sm, !first, s);
        else
            e = launch_fused_batch(p->d_jobs, p->d_chunks + b, n, acc, acc8, g, p->tune.ctas_per_sm,
                                   p->tune.warps_per_cta, p->tune.blocks_per_thread, !first, s);
        first = false;
    }
    if (e == cudaSuccess) e = launch_sse576_to_double(sse, p->nimages, s, sse8);
    return e;
}

rdct_status check_sse_args(const char *what, double *sse, double *sse8) {
    if (!sse) return set_error(RDCT_ERR_ARG, std::string(what) + ": null argument");
    if (reinterpret_cast<uintptr_t>(sse) % 8 || reinterpret_cast<uintptr_t>(sse8) % 8)
        return set_error(RDCT_ERR_ARG, std::string(what) + ": misaligned sse");
    if (sse8 == sse) return set_error(RDCT_ERR_ARG, std::string(what) + ": sse and sse_u8 must be different arrays");
    return RDCT_OK;
}

std::mutex g_tune_mu;
std::map<std::string, rdct_tune> g_tune_cache;

// The GPU model a tune was measured on (name, compute capability, SM count;
// not the device index), so that a saved cache applies to any device of that
// model.  Characters that would need escaping in the cache file are replaced.
std::string gpu_identity() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "nodev";
    }
    std::string name = prop.name;
    for (char &c : name)
        if (c == '"' || c == '\\' || c == ':' || (unsigned char)c < 32) c = '_';
    return name + "/sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "/" +
           std::to_string(prop.multiProcessorCount);
}

std::string shape_key(const rdct_job *jobs, int32_t njobs) {
    // shape class: job count, total blocks (log2 bucket) and blocks per r class
    int64_t blocks = 0;
    int64_t per_class[3] = {0};
    for (int32_t i = 0; i < njobs; ++i) {
        const int64_t b = (int64_t)(jobs[i].src.w / 8) * (jobs[i].src.h / 8);
        blocks += b;
        const int d = diag_class_host(jobs[i].r);
        per_class[d <= 5 ? 0 : (d <= 8 ? 1 : 2)] += b;
    }
    std::string k = gpu_identity() + ":n" + std::to_string(njobs);
    int lg = 0;
    while ((int64_t)1 << (lg + 1) <= blocks) ++lg;
    k += ":b" + std::to_string(lg);
    for (int c = 0; c < 3; ++c) k += ":" + std::to_string(blocks ? (int)(10 * per_class[c] / blocks) : 0);
    return k;
}

}  // namespace

extern "C" {

rdct_status rdct_batch_plan_create(const rdct_job *jobs, int32_t njobs, int32_t nimages, const rdct_tune *tune,
                                   rdct_plan **plan) {
    if (!plan) return set_error(RDCT_ERR_ARG, "rdct_batch_plan_create: null plan");
    *plan = nullptr;
    rdct_status st = validate_jobs(jobs, njobs, nimages);
    if (st) return st;
    rdct_tune t = default_tune();
    bool balance = false;
    if (tune) {
        t = *tune;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(shape_key(jobs, njobs));
        if (it != g_tune_cache.end()) t = it->second;
        else balance = true;
    }
    st = validate_tune(t);
    if (st) return st;
    rdct_plan *p = new (std::nothrow) rdct_plan();
    if (!p) return set_error(RDCT_ERR_OOM, "rdct_batch_plan_create: host allocation failed");
    p->nimages = nimages;
    p->tune = t;
    p->balance_chunks = balance;
    cudaGetDevice(&p->device);
    build_tables(p, jobs, njobs);
    const size_t jb = p->jobs.size() * sizeof(JobDesc), cb = p->chunks.size() * sizeof(Chunk);
    cudaError_t e = cudaSuccess;
    if (jb) e = cudaMalloc(&p->d_jobs, jb);
    if (e == cudaSuccess && cb) e = cudaMalloc(&p->d_chunks, cb);
    if (e != cudaSuccess) {
        rdct_batch_plan_destroy(p);
        return set_error(RDCT_ERR_OOM, "rdct_batch_plan_create: device table allocation failed");
    }
    if (jb) e = cudaMemcpy(p->d_jobs, p->jobs.data(), jb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && cb) e = cudaMemcpy(p->d_chunks, p->chunks.data(), cb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->tma) {
        e = cudaMalloc(&p->d_maps, p->maps.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->d_maps, p->maps.data(), p->maps.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);

    if (e != cudaSuccess) {
        rdct_batch_plan_destroy(p);
        return cuda_error(e, "rdct_batch_plan_create");
    }
    *plan = p;
    return RDCT_OK;
}

rdct_status rdct_batch_run(rdct_plan *p, double *sse, double *sse_u8, rdct_stream stream) {
    if (!p) return set_error(RDCT_ERR_ARG, "rdct_batch_run: null argument");
    rdct_status st = check_sse_args("rdct_batch_run", sse, sse_u8);
    if (st) return st;
    std::lock_guard<std::mutex> lk(p->mu);
    if (!p->exec || p->exec_sse != sse || p->exec_sse8 != sse_u8) {
        if (p->exec) {
            cudaGraphExecDestroy(p->exec);
            p->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        RDCT_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_batch(p, sse, sse_u8, p->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_error(e, "rdct_batch_run: capture");
        }
        if (e2 != cudaSuccess) return cuda_error(e2, "rdct_batch_run: end capture");
        e = cudaGraphInstantiate(&p->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->exec = nullptr;
            return cuda_error(e, "rdct_batch_run: instantiate");
        }
        p->exec_sse = sse;
        p->exec_sse8 = sse_u8;
    }
    RDCT_CUDA_TRY(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    return RDCT_OK;
}

rdct_status rdct_batch_run_per_plane(rdct_plan *p, double *sse, double *sse_u8, rdct_stream stream) {
    if (!p) return set_error(RDCT_ERR_ARG, "rdct_batch_run_per_plane: null argument");
    rdct_status st = check_sse_args("rdct_batch_run_per_plane", sse, sse_u8);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RDCT_CUDA_TRY(cudaMemsetAsync(sse, 0, (size_t)p->nimages * sizeof(double), s));
    if (sse_u8) RDCT_CUDA_TRY(cudaMemsetAsync(sse_u8, 0, (size_t)p->nimages * sizeof(double), s));
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(sse);
    unsigned long long *acc8 = reinterpret_cast<unsigned long long *>(sse_u8);
    for (const JobDesc &j : p->jobs_pp)
        RDCT_CUDA_TRY(launch_fused_single(j, RDCT_KIND_RDCT, acc + j.image, acc8 ? acc8 + j.image : nullptr, 0, 8, s));
    RDCT_CUDA_TRY(launch_sse576_to_double(sse, p->nimages, s, sse_u8));
    return RDCT_OK;
}

rdct_status rdct_batch_plan_kernels(const rdct_plan *p, int32_t *kernels_per_run) {
    if (!p || !kernels_per_run) return set_error(RDCT_ERR_ARG, "rdct_batch_plan_kernels: null argument");
    int32_t k = 1;  // the in-place 576*SSE -> SSE conversion
    for (int g = 0; g < 2 * kBatchGroups; ++g) k += p->group_begin[g + 1] > p->group_begin[g] ? 1 : 0;
    *kernels_per_run = k;
    return RDCT_OK;
}

rdct_status rdct_batch_plan_get_tune(const rdct_plan *p, rdct_tune *tune) {
    if (!p || !tune) return set_error(RDCT_ERR_ARG, "rdct_batch_plan_get_tune: null argument");
    *tune = p->tune;
    return RDCT_OK;
}

rdct_status rdct_batch_plan_destroy(rdct_plan *p) {
    if (!p) return RDCT_OK;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->cap_stream) {
        cudaStreamSynchronize(p->cap_stream);
        cudaStreamDestroy(p->cap_stream);
    }
    if (p->d_jobs) cudaFree(p->d_jobs);
    if (p->d_chunks) cudaFree(p->d_chunks);
    if (p->d_maps) cudaFree(p->d_maps);
    delete p;
    return RDCT_OK;
}

rdct_status rdct_autotune(const rdct_job *jobs, int32_t njobs, int32_t nimages, rdct_tune *best, rdct_stream stream) {
    if (!best) return set_error(RDCT_ERR_ARG, "rdct_autotune: null result");
    rdct_status st = validate_jobs(jobs, njobs, nimages);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *sse = nullptr;
    if (cudaMalloc(&sse, (size_t)(nimages > 0 ? nimages : 1) * sizeof(double)) != cudaSuccess)
        return set_error(RDCT_ERR_OOM, "rdct_autotune: scratch allocation failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaFree(sse);
        return set_error(RDCT_ERR_CUDA, "rdct_autotune: event creation failed");
    }
    // the default first, so that every other candidate is measured against it
    std::vector<rdct_tune> cands{default_tune()};
    for (int staging : {0, 1})
        for (int ctas : {0, 3, 4})
            for (int items : {4, 8, 16, 32}) {
                rdct_tune t = default_tune();
                t.ctas_per_sm = ctas;
                t.items_per_chunk = items;
                t.staging = staging;
                if (!same_tune(t, cands[0])) cands.push_back(t);
            }
    for (int items : {8, 16}) {  // the scalar kernel (one block per thread)
        rdct_tune t = default_tune();
        t.warps_per_cta = 8;
        t.blocks_per_thread = 1;
        t.items_per_chunk = items;
        cands.push_back(t);
    }
    // median of `reps` timed runs; a candidate whose runs spread by more than
    // 5% is measured once more, and dropped if it is still that noisy
    auto measure = [&](rdct_plan *p, float *median) -> bool {
        constexpr int reps = 5;
        for (int attempt = 0; attempt < 2; ++attempt) {
            std::vector<float> t;
            for (int k = 0; k < reps; ++k) {
                cudaEventRecord(e0, s);
                if (rdct_batch_run(p, sse, nullptr, s) != RDCT_OK) return false;
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) return false;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t.push_back(ms);
            }
            std::sort(t.begin(), t.end());
            *median = t[reps / 2];
            if (t.back() <= 1.05f * t.front()) return true;
        }
        *median = -1.0f;  // too noisy to rank
        return true;
    };
    float best_ms = 1e30f, default_ms = -1.0f;
    rdct_tune best_t = default_tune();
    rdct_status result = RDCT_OK;
    for (size_t c = 0; c < cands.size(); ++c) {
        const rdct_tune &t = cands[c];
        rdct_plan *p = nullptr;
        st = rdct_batch_plan_create(jobs, njobs, nimages, &t, &p);
        if (st) {
            result = st;
            break;
        }
        bool ok = rdct_batch_run(p, sse, nullptr, s) == RDCT_OK;  // capture + warm-up
        ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
        float med = -1.0f;
        ok = ok && measure(p, &med);
        rdct_batch_plan_destroy(p);
        if (!ok) {
            result = set_error(RDCT_ERR_CUDA, "rdct_autotune: a candidate failed to run");
            break;
        }
        if (c == 0) default_ms = med;
        if (med > 0.0f && med < best_ms) {
            best_ms = med;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sse);
    if (result != RDCT_OK) return result;
    // keep the default unless a candidate is clearly faster
    if (default_ms > 0.0f && best_ms > 0.99f * default_ms) best_t = default_tune();
    *best = best_t;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[shape_key(jobs, njobs)] = best_t;
    return RDCT_OK;
}

rdct_status rdct_autotune_cache_save(const char *path) {
    if (!path) return set_error(RDCT_ERR_ARG, "rdct_autotune_cache_save: null path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return set_error(RDCT_ERR_ARG, std::string("rdct_autotune_cache_save: cannot write ") + path);
    for (const auto &kv : g_tune_cache) {
        const rdct_tune &t = kv.second;
        std::fprintf(f,
                     "{\"key\": \"%s\", \"warps_per_cta\": %d, \"ctas_per_sm\": %d, \"items_per_chunk\": %d, "
                     "\"blocks_per_thread\": %d, \"staging\": %d}\n",
                     kv.first.c_str(), t.warps_per_cta, t.ctas_per_sm, t.items_per_chunk, t.blocks_per_thread,
                     t.staging);
    }
    const bool ok = std::fflush(f) == 0;
    std::fclose(f);
    if (!ok) return set_error(RDCT_ERR_ARG, std::string("rdct_autotune_cache_save: write failed: ") + path);
    return RDCT_OK;
}

rdct_status rdct_autotune_cache_load(const char *path, int32_t *loaded) {
    if (!path) return set_error(RDCT_ERR_ARG, "rdct_autotune_cache_load: null path");
    FILE *f = std::fopen(path, "r");
    if (!f) return set_error(RDCT_ERR_NOT_FOUND, std::string("rdct_autotune_cache_load: cannot read ") + path);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int32_t n = 0;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        char key[512];
        rdct_tune t{};
        int used = 0;
        // only the exact form rdct_autotune_cache_save writes; anything else is skipped
        if (std::sscanf(line,
                        "{\"key\": \"%511[^\"]\", \"warps_per_cta\": %d, \"ctas_per_sm\": %d, \"items_per_chunk\": "
                        "%d, \"blocks_per_thread\": %d, \"staging\": %d}%n",
                        key, &t.warps_per_cta, &t.ctas_per_sm, &t.items_per_chunk, &t.blocks_per_thread, &t.staging,
                        &used) != 6 ||
            used == 0)
            continue;
        if (validate_tune(t) != RDCT_OK) continue;
        g_tune_cache[key] = t;
        ++n;
    }
    std::fclose(f);
    if (loaded) *loaded = n;
    return RDCT_OK;
}

rdct_status rdct_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
    return RDCT_OK;
}

}  // extern "C"
