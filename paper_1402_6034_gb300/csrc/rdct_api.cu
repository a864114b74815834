// rdct_api.cu -- the C-ABI entry points for the method's steps (Sec. 2-3 of
// Cintra & Bayer): argument validation, constant set-up and launches.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rdct_device.cuh"
#include "rdct_internal.h"

namespace rdct {

static thread_local std::string g_last_error;

rdct_status set_error(rdct_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

rdct_status cuda_error(cudaError_t e, const char *what) {
    return set_error(RDCT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

int sm_count() {
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

// Exact DCT (Sec. 2 "standard DCT matrix"): C[k][n] = a_k cos(pi (2n+1) k / 16).
DctConsts make_dct_consts() {
    DctConsts c{};
    const double pi = std::acos(-1.0);
    for (int k = 0; k < 8; ++k)
        for (int n = 0; n < 8; ++n)
            c.c[k * 8 + n] = (float)((k == 0 ? std::sqrt(0.125) : 0.5) * std::cos(pi * (2 * n + 1) * k / 16.0));
    return c;
}

// d_i d_j = 1 / sqrt(g_i g_j), the orthonormal scaling of C0 coefficients.
ScaleConsts make_scale_consts() {
    ScaleConsts s{};
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) s.dd[i * 8 + j] = (float)(1.0 / std::sqrt((double)(gram(i) * gram(j))));
    return s;
}

int diag_class_host(int r) { return diag_class(r); }

static int align_of(const void *p, int64_t pitch) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if ((a % 16) == 0 && (pitch % 16) == 0) return 16;
    if ((a % 8) == 0 && (pitch % 8) == 0) return 8;
    return 1;
}

rdct_status validate_plane(const rdct_plane *p, const char *what) {
    if (!p) return set_error(RDCT_ERR_ARG, std::string(what) + ": null plane");
    if (!p->ptr) return set_error(RDCT_ERR_ARG, std::string(what) + ": null pixel pointer");
    if (p->w <= 0 || p->h <= 0 || (p->w % 8) || (p->h % 8))
        return set_error(RDCT_ERR_SHAPE, std::string(what) + ": width and height must be positive multiples of 8 (got " +
                                             std::to_string(p->w) + "x" + std::to_string(p->h) + ")");
    if (p->pitch < p->w) return set_error(RDCT_ERR_SHAPE, std::string(what) + ": pitch smaller than width");
    // 576 * SSE of a plane must stay below 2^63 (at most 576 * 64 * 255^2 per block)
    if ((int64_t)(p->w / 8) * (p->h / 8) > (int64_t)1 << 30)
        return set_error(RDCT_ERR_TOO_LARGE, std::string(what) + ": plane too large");
    return RDCT_OK;
}

JobDesc make_job(const rdct_plane &src, uint8_t *dst, int64_t dst_pitch, float *dstf, int64_t dstf_pitch, int32_t r,
                 int32_t image, int bpt) {
    JobDesc j{};
    j.src = src.ptr;
    j.dst = dst;
    j.dstf = dstf;
    j.src_pitch = src.pitch;
    j.dst_pitch = dst_pitch;
    j.dstf_pitch = dstf_pitch;
    j.nbw = src.w / 8;
    j.nbh = src.h / 8;
    j.r = r;
    j.image = image;
    const int per = 32 * bpt;
    j.segs = (j.nbw + per - 1) / per;
    j.align = align_of(src.ptr, src.pitch);
    j.dalign = dst ? align_of(dst, dst_pitch) : 16;
    return j;
}

}  // namespace rdct

using namespace rdct;

static rdct_status finish_launch(cudaError_t e, const char *what) {
    if (e != cudaSuccess) return cuda_error(e, what);
    return RDCT_OK;
}

static rdct_status validate_out(const rdct_out *out, int32_t w, int32_t h) {
    if (!out) return RDCT_OK;
    if (out->u8 && out->pitch < w) return set_error(RDCT_ERR_SHAPE, "out: u8 pitch smaller than width");
    if (out->f32 && out->pitch_f32 < w) return set_error(RDCT_ERR_SHAPE, "out: f32 pitch smaller than width");
    (void)h;
    return RDCT_OK;
}

extern "C" {

const char *rdct_status_string(rdct_status s) {
    switch (s) {
        case RDCT_OK: return "ok";
        case RDCT_ERR_ARG: return "invalid argument";
        case RDCT_ERR_SHAPE: return "invalid shape";
        case RDCT_ERR_OOM: return "out of memory";
        case RDCT_ERR_TOO_LARGE: return "too large";
        case RDCT_ERR_CUDA: return "CUDA error";
        case RDCT_ERR_TIMEOUT: return "timeout";
        case RDCT_ERR_BUSY: return "busy";
        case RDCT_ERR_NOT_FOUND: return "not found";
        case RDCT_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

size_t rdct_last_error(char *buf, size_t cap) {
    const std::string &m = g_last_error;
    if (buf && cap) {
        const size_t n = m.size() < cap - 1 ? m.size() : cap - 1;
        std::memcpy(buf, m.data(), n);
        buf[n] = 0;
    }
    return m.size();
}

int32_t rdct_version(void) { return 1 * 10000 + 0 * 100 + 0; }

rdct_status rdct_sync(rdct_stream stream) {
    RDCT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    RDCT_CUDA_TRY(cudaGetLastError());
    unsigned int (*const takers[])() = {
        take_tma_timeouts_r0,  take_tma_timeouts_r1,  take_tma_timeouts_r2,  take_tma_timeouts_r3,
        take_tma_timeouts_r4,  take_tma_timeouts_r5,  take_tma_timeouts_r6,  take_tma_timeouts_r7,
        take_tma_timeouts_r8,  take_tma_timeouts_r9,  take_tma_timeouts_r10, take_tma_timeouts_r11,
        take_tma_timeouts_r12, take_tma_timeouts_r13, take_tma_timeouts_r14, take_tma_timeouts_r15};
    unsigned int t = 0;
    for (auto take : takers) t += take();
    const unsigned int ts = take_sweep_tc_timeouts();
    if (ts)
        return set_error(RDCT_ERR_TIMEOUT, "rdct_sync: " + std::to_string(ts) +
                                               " waits of the tensor-core sweep for its MMAs ran out; those groups "
                                               "stopped early and the sweep results are incomplete");
    if (t)
        return set_error(RDCT_ERR_TIMEOUT, "rdct_sync: " + std::to_string(t) +
                                               " TMA waits for a staged box ran out; the launches that hit them "
                                               "stopped early and their results are incomplete");
    return RDCT_OK;
}

rdct_status rdct_forward(const rdct_plane *src, int32_t *Y, rdct_stream stream) {
    rdct_status st = validate_plane(src, "rdct_forward");
    if (st) return st;
    if (!Y) return set_error(RDCT_ERR_ARG, "rdct_forward: null Y");
    if (reinterpret_cast<uintptr_t>(Y) % 16) return set_error(RDCT_ERR_ARG, "rdct_forward: Y must be 16-byte aligned");
    const JobDesc job = make_job(*src, nullptr, 0, nullptr, 0, 64, 0, 1);
    return finish_launch(launch_forward(job, Y, (cudaStream_t)stream), "rdct_forward");
}

rdct_status rdct_forward_f32(const rdct_plane *src, rdct_kind kind, float *Y, rdct_stream stream) {
    rdct_status st = validate_plane(src, "rdct_forward_f32");
    if (st) return st;
    if (!Y) return set_error(RDCT_ERR_ARG, "rdct_forward_f32: null Y");
    if (kind != RDCT_KIND_RDCT && kind != RDCT_KIND_DCT) return set_error(RDCT_ERR_ARG, "rdct_forward_f32: bad kind");
    if (reinterpret_cast<uintptr_t>(Y) % 16)
        return set_error(RDCT_ERR_ARG, "rdct_forward_f32: Y must be 16-byte aligned");
    const JobDesc job = make_job(*src, nullptr, 0, nullptr, 0, 64, 0, 1);
    return finish_launch(launch_forward_f32(job, (int)kind, Y, (cudaStream_t)stream), "rdct_forward_f32");
}

rdct_status rdct_compress(const int32_t *Y, int64_t nblocks, int32_t r, float *Yc, rdct_stream stream) {
    if (!Y || !Yc || nblocks < 0) return set_error(RDCT_ERR_ARG, "rdct_compress: null pointer or negative count");
    if (r < 1 || r > 64) return set_error(RDCT_ERR_ARG, "rdct_compress: r must be in 1..64");
    if (nblocks == 0) return RDCT_OK;
    return finish_launch(launch_compress(Y, nblocks, r, Yc, (cudaStream_t)stream), "rdct_compress");
}

rdct_status rdct_inverse(const float *Yc, int64_t nbw, int64_t nbh, int32_t r, rdct_kind kind, const rdct_out *out,
                         rdct_stream stream) {
    if (!Yc || !out || nbw < 0 || nbh < 0) return set_error(RDCT_ERR_ARG, "rdct_inverse: null pointer or negative size");
    if (r < 1 || r > 64) return set_error(RDCT_ERR_ARG, "rdct_inverse: r must be in 1..64");
    if (kind != RDCT_KIND_RDCT && kind != RDCT_KIND_DCT) return set_error(RDCT_ERR_ARG, "rdct_inverse: bad kind");
    if (!out->u8 && !out->f32) return set_error(RDCT_ERR_ARG, "rdct_inverse: no output");
    rdct_status st = validate_out(out, (int32_t)(nbw * 8), (int32_t)(nbh * 8));
    if (st) return st;
    if (nbw == 0 || nbh == 0) return RDCT_OK;
    return finish_launch(launch_inverse(Yc, nbw, nbh, r, (int)kind, out->u8, out->pitch, out->f32, out->pitch_f32,
                                        (cudaStream_t)stream),
                         "rdct_inverse");
}

rdct_status rdct_mse_psnr(const rdct_plane *ref, const rdct_out *rec, double *mse, double *psnr, rdct_stream stream) {
    rdct_status st = validate_plane(ref, "rdct_mse_psnr");
    if (st) return st;
    if (!rec || (!rec->u8 && !rec->f32) || !mse || !psnr)
        return set_error(RDCT_ERR_ARG, "rdct_mse_psnr: null reconstruction or output");
    st = validate_out(rec, ref->w, ref->h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, 16, s);
    if (e != cudaSuccess) return set_error(RDCT_ERR_OOM, "rdct_mse_psnr: scratch allocation failed");
    unsigned long long *acc_u = reinterpret_cast<unsigned long long *>(scratch);
    double *acc_f = reinterpret_cast<double *>(scratch) + 1;
    e = cudaMemsetAsync(scratch, 0, 16, s);
    const JobDesc job = make_job(*ref, nullptr, 0, nullptr, 0, 64, 0, 1);
    if (e == cudaSuccess) e = launch_sse(job, rec->u8, rec->pitch, rec->u8 ? nullptr : rec->f32, rec->pitch_f32, acc_u, acc_f, s);
    if (e == cudaSuccess)
        e = launch_mse_finalize(acc_u, acc_f, rec->u8 ? 1 : 0, (double)ref->w * (double)ref->h, mse, psnr, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_error(e, "rdct_mse_psnr");
    if (e2 != cudaSuccess) return cuda_error(e2, "rdct_mse_psnr: free");
    return RDCT_OK;
}

rdct_status rdct_fused(const rdct_plane *src, int32_t r, rdct_kind kind, const rdct_out *out, double *sse,
                       double *sse_u8, rdct_stream stream) {
    rdct_status st = validate_plane(src, "rdct_fused");
    if (st) return st;
    if (r < 1 || r > 64) return set_error(RDCT_ERR_ARG, "rdct_fused: r must be in 1..64");
    if (kind != RDCT_KIND_RDCT && kind != RDCT_KIND_DCT) return set_error(RDCT_ERR_ARG, "rdct_fused: bad kind");
    if (!sse) return set_error(RDCT_ERR_ARG, "rdct_fused: null sse");
    if (reinterpret_cast<uintptr_t>(sse) % 8) return set_error(RDCT_ERR_ARG, "rdct_fused: sse must be 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(sse_u8) % 8)
        return set_error(RDCT_ERR_ARG, "rdct_fused: sse_u8 must be 8-byte aligned");
    if (sse_u8 == sse) return set_error(RDCT_ERR_ARG, "rdct_fused: sse and sse_u8 must be different slots");
    st = validate_out(out, src->w, src->h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const JobDesc job = make_job(*src, out ? out->u8 : nullptr, out ? out->pitch : 0, out ? out->f32 : nullptr,
                                 out ? out->pitch_f32 : 0, r, 0, 1);
    unsigned long long *acc8 = reinterpret_cast<unsigned long long *>(sse_u8);
    RDCT_CUDA_TRY(cudaMemsetAsync(sse, 0, sizeof(double), s));
    if (acc8) RDCT_CUDA_TRY(cudaMemsetAsync(acc8, 0, sizeof(double), s));
    RDCT_CUDA_TRY(launch_fused_single(job, (int)kind, sse, acc8, 0, 8, s));
    if (kind == RDCT_KIND_RDCT || acc8)
        RDCT_CUDA_TRY(launch_sse576_to_double(kind == RDCT_KIND_RDCT ? sse : nullptr, 1, s, acc8));
    return RDCT_OK;
}

rdct_status rdct_sweep(const rdct_plane *planes, int32_t n, rdct_kind kind, double *sse_by_r, rdct_stream stream) {
    if (!planes || !sse_by_r || n < 0) return set_error(RDCT_ERR_ARG, "rdct_sweep: null pointer or negative count");
    if (kind != RDCT_KIND_RDCT && kind != RDCT_KIND_DCT) return set_error(RDCT_ERR_ARG, "rdct_sweep: bad kind");
    if (reinterpret_cast<uintptr_t>(sse_by_r) % 8) return set_error(RDCT_ERR_ARG, "rdct_sweep: misaligned output");
    if (n == 0) return RDCT_OK;
    int64_t nchunks = 0, ntiles = 0;
    for (int32_t i = 0; i < n; ++i) {
        rdct_status st = validate_plane(&planes[i], "rdct_sweep");
        if (st) return st;
        nchunks += sweep_chunk_count(planes[i]);
        ntiles += sweep_tiles_of(planes[i]);
    }
    if (nchunks > INT32_MAX || ntiles > INT32_MAX)
        return set_error(RDCT_ERR_TOO_LARGE, "rdct_sweep: too many strips in one call");
    cudaStream_t s = (cudaStream_t)stream;
    // (the tiled pass needs the job table alone)
    const size_t jb = ((size_t)n * sizeof(JobDesc) + 255) & ~(size_t)255,
                 cb = sweep_is_tiled((int)kind) ? 0 : (size_t)nchunks * sizeof(Chunk);
    void *tables = nullptr;
    if (cudaMallocAsync(&tables, jb + cb, s) != cudaSuccess)
        return set_error(RDCT_ERR_OOM, "rdct_sweep: table allocation failed");
    JobDesc *jd = reinterpret_cast<JobDesc *>(tables);
    Chunk *cd = reinterpret_cast<Chunk *>(reinterpret_cast<char *>(tables) + jb);
    cudaError_t e = build_sweep_tables(planes, n, sweep_is_tiled((int)kind), jd, cd, sse_by_r, s);
    if (e == cudaSuccess) e = launch_sweep(jd, cd, (int32_t)nchunks, (int)kind, sse_by_r, n, (int32_t)ntiles, s);
    if (e == cudaSuccess) e = launch_sweep_finalize(sse_by_r, n, (int)kind, s);
    cudaError_t e2 = cudaFreeAsync(tables, s);
    if (e != cudaSuccess) return cuda_error(e, "rdct_sweep");
    if (e2 != cudaSuccess) return cuda_error(e2, "rdct_sweep: free");
    return RDCT_OK;
}

}  // extern "C"
