// rdct_kernels.cu -- CUDA kernels of the RDCT path for sm_103a.
//
// Sec. 3 of Cintra & Bayer: every 8x8 block A of an image is transformed as
// T A T^T, the first r coefficients of the zigzag sequence are kept, the block
// is reconstructed with the inverse and the error is measured.  With the
// proposed T = C_orth = S C0 (Sec. 2) the transform is additions only and the
// diagonal S is folded into the compression step (Sec. 2): this file does the
// additions in int32 / exact FP32 registers and the scaling as integer weights.
//
// Mapping: one thread owns one 8x8 block; a warp owns a strip of 32
// horizontally adjacent blocks of one block row, so every row load of a warp
// is 256 contiguous bytes.  Kernels are persistent (grid-stride over strips).
#include <cuda_runtime.h>

#include <cstdint>

#include "rdct_blocks.cuh"

namespace rdct {

// In place: uint64 576 * SSE -> double SSE (slots not nullptr), and uint64
// squared errors of 8-bit reconstructions -> double (slots8 not nullptr).
__global__ void sse576_to_double_kernel(void *slots, void *slots8, int32_t n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        if (slots != nullptr) {
            const unsigned long long u = reinterpret_cast<unsigned long long *>(slots)[i];
            reinterpret_cast<double *>(slots)[i] = (double)u / 576.0;
        }
        if (slots8 != nullptr) {
            const unsigned long long v = reinterpret_cast<unsigned long long *>(slots8)[i];
            reinterpret_cast<double *>(slots8)[i] = (double)v;
        }
    }
}

// ------------------------------------------------------- forward kernels

__global__ void __launch_bounds__(256) forward_kernel(const JobDesc job, int32_t *__restrict__ Y) {
    const int64_t nblocks = (int64_t)job.nbw * job.nbh;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int by = (int)(b / job.nbw), bx = (int)(b - (int64_t)by * job.nbw);
        uint32_t w[16];
        load_block(job.src + (int64_t)by * 8 * job.src_pitch + (int64_t)bx * 8, job.src_pitch, job.align, w);
        int Yb[8][8];
        forward_c0(w, Yb);
        int4 *out = reinterpret_cast<int4 *>(Y + b * 64);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            __stcs(out + 2 * i, make_int4(Yb[i][0], Yb[i][1], Yb[i][2], Yb[i][3]));
            __stcs(out + 2 * i + 1, make_int4(Yb[i][4], Yb[i][5], Yb[i][6], Yb[i][7]));
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) forward_f32_kernel(const JobDesc job, float *__restrict__ Y,
                                                          const DctConsts C, const ScaleConsts S) {
    const int64_t nblocks = (int64_t)job.nbw * job.nbh;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int by = (int)(b / job.nbw), bx = (int)(b - (int64_t)by * job.nbw);
        uint32_t w[16];
        load_block(job.src + (int64_t)by * 8 * job.src_pitch + (int64_t)bx * 8, job.src_pitch, job.align, w);
        float Yf[8][8];
        if constexpr (KIND == RDCT_KIND_RDCT) {
            int Yb[8][8];
            forward_c0(w, Yb);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) Yf[i][j] = (float)Yb[i][j] * S.dd[i * 8 + j];
        } else {
            float A[8][8];
            forward_dct(w, Yf, A, C);
        }
        float4 *out = reinterpret_cast<float4 *>(Y + b * 64);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            __stcs(out + 2 * i, make_float4(Yf[i][0], Yf[i][1], Yf[i][2], Yf[i][3]));
            __stcs(out + 2 * i + 1, make_float4(Yf[i][4], Yf[i][5], Yf[i][6], Yf[i][7]));
        }
    }
}

// ------------------------------------------------- compress / inverse kernels

struct ZigzagTable {
    int8_t pos[64];
};
__host__ ZigzagTable make_zigzag_table() {
    ZigzagTable t{};
    for (int k = 0; k < 64; ++k) t.pos[k] = (int8_t)zz_pos(k);
    return t;
}

// Yc[b][k] = d_i d_j Y[b][i][j] for the k-th zigzag position (i, j), k < r.
__global__ void compress_kernel(const int32_t *__restrict__ Y, int64_t nblocks, int32_t r, float *__restrict__ Yc,
                                const ZigzagTable zz, const ScaleConsts S) {
    const int64_t total = nblocks * r;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / r;
        const int k = (int)(t - b * r);
        const int p = zz.pos[k];
        Yc[t] = (float)__ldg(Y + b * 64 + p) * S.dd[p];
    }
}

// Xhat = C0^T (S Yhat S) C0 for kind RDCT, C^T Yhat C for kind DCT; FP32.
template <int KIND>
__global__ void __launch_bounds__(256) inverse_kernel(const float *__restrict__ Yc, int64_t nbw, int64_t nbh,
                                                      int32_t r, uint8_t *u8, int64_t pitch, float *f32,
                                                      int64_t pitch_f32, const ZigzagTable zz, const ScaleConsts S,
                                                      const DctConsts C) {
    const int64_t nblocks = nbw * nbh;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t by = b / nbw, bx = b - by * nbw;
        float Z[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) Z[i][j] = 0.0f;
        const float *src = Yc + b * r;
        static_for<0, 64>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int k = zz_rank(q >> 3, q & 7);
            if (k < r) {
                const float v = __ldg(src + k);
                Z[q >> 3][q & 7] = (KIND == RDCT_KIND_RDCT) ? v * S.dd[q] : v;
            }
        });
        float U[8][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float in[8], out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) in[i] = Z[i][j];
            if constexpr (KIND == RDCT_KIND_RDCT) c0t_inverse<0xFFu>(in, out);
            else dct_inv8<0xFFu>(in, out, C);
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = out[i];
        }
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            float X[8];
            if constexpr (KIND == RDCT_KIND_RDCT) c0t_inverse<0xFFu>(U[n], X);
            else dct_inv8<0xFFu>(U[n], X, C);
            const int64_t row = by * 8 + n;
            if (u8) {
                uint8_t *p = u8 + row * pitch + bx * 8;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int q = q_of(X[m]);
                    p[m] = (uint8_t)(q < 0 ? 0 : (q > 255 ? 255 : q));
                }
            }
            if (f32) {
                float *p = f32 + row * pitch_f32 + bx * 8;
#pragma unroll
                for (int m = 0; m < 8; ++m) p[m] = X[m];
            }
        }
    }
}

// ------------------------------------------------------------ SSE / PSNR

__global__ void __launch_bounds__(256) sse_kernel(const JobDesc ref, const uint8_t *__restrict__ rec_u8,
                                                  int64_t rec_pitch, const float *__restrict__ rec_f32,
                                                  int64_t rec_pitch_f32, unsigned long long *acc_u64,
                                                  double *acc_f64) {
    const int64_t groups_per_row = ref.nbw;  // 8-pixel groups
    const int64_t total = groups_per_row * (int64_t)ref.nbh * 8;
    unsigned long long su = 0;
    double sf = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = g / groups_per_row, x = (g - y * groups_per_row) * 8;
        const uint8_t *a = ref.src + y * ref.src_pitch + x;
        if (rec_u8) {
            const uint8_t *b = rec_u8 + y * rec_pitch + x;
            unsigned s = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int d = (int)a[k] - (int)b[k];
                s += (unsigned)(d * d);
            }
            su += s;
        } else {
            const float *b = rec_f32 + y * rec_pitch_f32 + x;
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float d = b[k] - (float)a[k];
                s = __fmaf_rn(d, d, s);
            }
            sf += (double)s;
        }
    }
    const int lane = threadIdx.x & 31;
    if (rec_u8) {
        su = warp_sum_u64(su);
        if (lane == 0 && su) atomicAdd(acc_u64, su);
    } else {
        sf = warp_sum_f64(sf);
        if (lane == 0 && sf != 0.0) atomicAdd(acc_f64, sf);
    }
}

__global__ void mse_finalize_kernel(const unsigned long long *acc_u64, const double *acc_f64, int use_u64,
                                    double nsamples, double *mse, double *psnr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double s = use_u64 ? (double)*acc_u64 : *acc_f64;
        const double m = s / nsamples;
        *mse = m;
        *psnr = (m == 0.0) ? __longlong_as_double(0x7ff0000000000000LL) : 10.0 * log10(255.0 * 255.0 / m);
    }
}

// ------------------------------------------------------------------ sweep

// In place: 64 zigzag bins per plane -> SSE(r) = sum of bins k >= r, r = 1..64.
// One warp per plane: lane l holds bins 2l and 2l+1; a suffix scan over the
// warp gives every tail sum.
__global__ void sweep_finalize_kernel(double *out, int32_t nplanes, int kind) {
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= nplanes) return;
    double *o = out + (int64_t)warp * 64;
    if (kind == RDCT_KIND_RDCT) {
        const unsigned long long *u = reinterpret_cast<const unsigned long long *>(o);
        const unsigned long long b0 = u[2 * lane], b1 = u[2 * lane + 1];
        unsigned long long t = b0 + b1;  // suffix sum over lanes >= lane
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long v = __shfl_down_sync(0xffffffffu, t, d);
            if (lane + d < 32) t += v;
        }
        __syncwarp();
        // SSE(r) keeps ranks < r: r = 2l+1 drops bins >= 2l+1, r = 2l+2 drops bins >= 2l+2
        o[2 * lane] = (double)(t - b0) / 576.0;
        o[2 * lane + 1] = (double)(t - b0 - b1) / 576.0;
    } else {
        const double b0 = o[2 * lane], b1 = o[2 * lane + 1];
        double t = b0 + b1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double v = __shfl_down_sync(0xffffffffu, t, d);
            if (lane + d < 32) t += v;
        }
        __syncwarp();
        // tails summed from the small end (lanes >= lane), so small bins are not lost
        o[2 * lane] = t - b0;
        o[2 * lane + 1] = t - b0 - b1;
    }
}

// ------------------------------------------------------------- launchers

static int grid_for(int64_t work_items, int threads, int ctas_per_sm = 4) {
    const int64_t need = (work_items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * ctas_per_sm;
    int64_t g = need < cap ? need : cap;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_forward(const JobDesc &job, int32_t *Y, cudaStream_t s) {
    const int64_t nb = (int64_t)job.nbw * job.nbh;
    forward_kernel<<<grid_for(nb, 256, 8), 256, 0, s>>>(job, Y);
    return cudaGetLastError();
}

cudaError_t launch_forward_f32(const JobDesc &job, int kind, float *Y, cudaStream_t s) {
    const int64_t nb = (int64_t)job.nbw * job.nbh;
    const DctConsts C = make_dct_consts();
    const ScaleConsts S = make_scale_consts();
    if (kind == RDCT_KIND_RDCT) forward_f32_kernel<RDCT_KIND_RDCT><<<grid_for(nb, 256, 8), 256, 0, s>>>(job, Y, C, S);
    else forward_f32_kernel<RDCT_KIND_DCT><<<grid_for(nb, 256, 8), 256, 0, s>>>(job, Y, C, S);
    return cudaGetLastError();
}

cudaError_t launch_compress(const int32_t *Y, int64_t nblocks, int32_t r, float *Yc, cudaStream_t s) {
    compress_kernel<<<grid_for(nblocks * r, 256, 16), 256, 0, s>>>(Y, nblocks, r, Yc, make_zigzag_table(),
                                                                   make_scale_consts());
    return cudaGetLastError();
}

cudaError_t launch_inverse(const float *Yc, int64_t nbw, int64_t nbh, int32_t r, int kind, uint8_t *u8, int64_t pitch,
                           float *f32, int64_t pitch_f32, cudaStream_t s) {
    const int64_t nb = nbw * nbh;
    const int g = grid_for(nb, 256, 8);
    if (kind == RDCT_KIND_RDCT)
        inverse_kernel<RDCT_KIND_RDCT><<<g, 256, 0, s>>>(Yc, nbw, nbh, r, u8, pitch, f32, pitch_f32,
                                                         make_zigzag_table(), make_scale_consts(), DctConsts{});
    else
        inverse_kernel<RDCT_KIND_DCT><<<g, 256, 0, s>>>(Yc, nbw, nbh, r, u8, pitch, f32, pitch_f32,
                                                        make_zigzag_table(), ScaleConsts{}, make_dct_consts());
    return cudaGetLastError();
}

cudaError_t launch_sse(const JobDesc &ref, const uint8_t *rec_u8, int64_t rec_pitch, const float *rec_f32,
                       int64_t rec_pitch_f32, unsigned long long *acc_u64, double *acc_f64, cudaStream_t s) {
    const int64_t groups = (int64_t)ref.nbw * ref.nbh * 8;
    sse_kernel<<<grid_for(groups, 256, 8), 256, 0, s>>>(ref, rec_u8, rec_pitch, rec_f32, rec_pitch_f32, acc_u64,
                                                         acc_f64);
    return cudaGetLastError();
}

cudaError_t launch_mse_finalize(const unsigned long long *acc_u64, const double *acc_f64, int use_u64,
                                double nsamples, double *mse, double *psnr, cudaStream_t s) {
    mse_finalize_kernel<<<1, 32, 0, s>>>(acc_u64, acc_f64, use_u64, nsamples, mse, psnr);
    return cudaGetLastError();
}

cudaError_t launch_sse576_to_double(void *slots, int32_t n, cudaStream_t s, void *slots8) {
    if (n <= 0) return cudaSuccess;
    sse576_to_double_kernel<<<(n + 255) / 256, 256, 0, s>>>(slots, slots8, n);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, int kind, double *out,
                         int32_t nplanes, cudaStream_t s) {
    (void)nplanes;
    if (nchunks <= 0) return cudaSuccess;
    return launch_sweep2(jobs, chunks, nchunks, kind, out, s);
}

cudaError_t launch_sweep_finalize(double *out, int32_t nplanes, int kind, cudaStream_t s) {
    if (nplanes <= 0) return cudaSuccess;
    sweep_finalize_kernel<<<(nplanes + 3) / 4, 128, 0, s>>>(out, nplanes, kind);
    return cudaGetLastError();
}

}  // namespace rdct
