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
    // launched as a programmatic dependent of the kernels that filled the slots
    asm volatile("griddepcontrol.wait;" ::: "memory");
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

// One warp per 32 consecutive blocks (block index b = by * nbw + bx, so their
// coefficients are one contiguous 8 KB run of Y): each lane transforms its
// block and writes its 64 values to the warp's shared-memory stage (16-byte
// words swizzled so that neither the writes nor the reads conflict on banks),
// and the warp then stores the run with every store instruction covering 512
// contiguous bytes.
constexpr int kFwdWarps = 4;

// Lane's block row i (8 values of 4 bytes) into the stage.
__device__ __forceinline__ void stage_row(int4 *st, int lane, int i, int4 lo, int4 hi) {
    st[lane * 16 + ((2 * i) ^ (lane & 7))] = lo;
    st[lane * 16 + ((2 * i + 1) ^ (lane & 7))] = hi;
}
// The warp's staged run (nvalid blocks of 256 bytes) to out.
__device__ __forceinline__ void store_run(const int4 *st, int4 *out, int64_t nvalid, int lane) {
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int j = k * 32 + lane;  // 16-byte word j of the run: block j / 16, word j % 16
        const int jb = j >> 4, jw = j & 15;
        if (jb < nvalid) __stcs(out + j, st[jb * 16 + (jw ^ (jb & 7))]);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kFwdWarps * 32) forward_kernel(const JobDesc job, int32_t *__restrict__ Y) {
    __shared__ int4 stage[kFwdWarps][32 * 16];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 *st = stage[wid];
    const int64_t nblocks = (int64_t)job.nbw * job.nbh;
    const int64_t step = (int64_t)gridDim.x * kFwdWarps * 32;
    for (int64_t b0 = ((int64_t)blockIdx.x * kFwdWarps + wid) * 32; b0 < nblocks; b0 += step) {
        const int64_t b = b0 + lane;
        if (b < nblocks) {
            const int64_t by = b / job.nbw, bx = b - by * job.nbw;
            uint32_t w[16];
            load_block(job.src + by * 8 * job.src_pitch + bx * 8, job.src_pitch, job.align, w);
            int Yb[8][8];
            forward_c0(w, Yb);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                stage_row(st, lane, i, make_int4(Yb[i][0], Yb[i][1], Yb[i][2], Yb[i][3]),
                          make_int4(Yb[i][4], Yb[i][5], Yb[i][6], Yb[i][7]));
        }
        store_run(st, reinterpret_cast<int4 *>(Y) + b0 * 16, nblocks - b0 < 32 ? nblocks - b0 : 32, lane);
    }
}

template <int KIND>
__global__ void __launch_bounds__(kFwdWarps * 32) forward_f32_kernel(const JobDesc job, float *__restrict__ Y,
                                                                     const DctConsts C, const ScaleConsts S) {
    __shared__ int4 stage[kFwdWarps][32 * 16];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 *st = stage[wid];
    const int64_t nblocks = (int64_t)job.nbw * job.nbh;
    const int64_t step = (int64_t)gridDim.x * kFwdWarps * 32;
    for (int64_t b0 = ((int64_t)blockIdx.x * kFwdWarps + wid) * 32; b0 < nblocks; b0 += step) {
        const int64_t b = b0 + lane;
        if (b < nblocks) {
            const int64_t by = b / job.nbw, bx = b - by * job.nbw;
            uint32_t w[16];
            load_block(job.src + by * 8 * job.src_pitch + bx * 8, job.src_pitch, job.align, w);
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
#pragma unroll
            for (int i = 0; i < 8; ++i)
                stage_row(st, lane, i,
                          make_int4(__float_as_int(Yf[i][0]), __float_as_int(Yf[i][1]), __float_as_int(Yf[i][2]),
                                    __float_as_int(Yf[i][3])),
                          make_int4(__float_as_int(Yf[i][4]), __float_as_int(Yf[i][5]), __float_as_int(Yf[i][6]),
                                    __float_as_int(Yf[i][7])));
        }
        store_run(st, reinterpret_cast<int4 *>(Y) + b0 * 16, nblocks - b0 < 32 ? nblocks - b0 : 32, lane);
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
// D: the anti-diagonal class of r (positions beyond it are zero and skipped).
// One thread per block; the coefficients are read through L1 (a warp's 32
// blocks are one contiguous run of 32 r floats), rows are stored 8 pixels (or
// 8 floats) at a time when the output allows it.
template <int KIND, int D>
__global__ void __launch_bounds__(256) inverse_kernel(const float *__restrict__ Yc, int64_t nbw, int64_t nbh,
                                                      int32_t r, uint8_t *u8, int64_t pitch, int u8_align,
                                                      float *f32, int64_t pitch_f32, const ScaleConsts S,
                                                      const DctConsts C) {
    const int64_t nblocks = nbw * nbh;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t by = b / nbw, bx = b - by * nbw;
        float Z[8][8];
        const float *src = Yc + b * r;
        static_for<0, 64>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int i = q >> 3, j = q & 7;
            if constexpr (i + j <= D) {
                constexpr int k = zz_rank(i, j);
                float v = 0.0f;
                if (i + j < D || k < r) v = __ldg(src + k);
                Z[i][j] = (KIND == RDCT_KIND_RDCT) ? v * S.dd[q] : v;
            } else {
                Z[i][j] = 0.0f;
            }
        });
        float U[8][8];
        static_for<0, 8>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr unsigned m = col_mask(D, j);
            float in[8], out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) in[i] = Z[i][j];
            if constexpr (m == 0u) {
#pragma unroll
                for (int i = 0; i < 8; ++i) out[i] = 0.0f;
            } else if constexpr (KIND == RDCT_KIND_RDCT) {
                c0t_inverse<m>(in, out);
            } else {
                dct_inv8<m>(in, out, C);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = out[i];
        });
        constexpr unsigned rm = row_mask(D);
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            float X[8];
            if constexpr (KIND == RDCT_KIND_RDCT) c0t_inverse<rm>(U[n], X);
            else dct_inv8<rm>(U[n], X, C);
            const int64_t row = by * 8 + n;
            if (u8) {
                int q[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) q[m] = q_of(X[m]);
                store_row_u8(u8 + row * pitch + bx * 8, u8_align, pack4_sat(q[0], q[1], q[2], q[3]),
                             pack4_sat(q[4], q[5], q[6], q[7]));
            }
            if (f32) store_row_f32(f32 + row * pitch_f32 + bx * 8, X);
        }
    }
}

// ------------------------------------------------------------ SSE / PSNR

// Squared error of a reconstruction against a plane.  One warp per row at a
// time, lanes stepping across it: V pixels per lane and step (16 when both
// planes start on 16-byte boundaries with 16-byte pitches, 8 when on 8-byte
// ones, else 1).  For uint8 reconstructions sum (a - b)^2 = sum a^2 + sum b^2
// - 2 sum a b is formed exactly from byte dot products.
template <int V>
__device__ __forceinline__ void load_px(const uint8_t *p, uint32_t (&w)[V / 4 > 0 ? V / 4 : 1]) {
    if constexpr (V == 16) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(p));
        w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    } else if constexpr (V == 8) {
        const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
        w[0] = v.x, w[1] = v.y;
    } else {
        w[0] = p[0];
    }
}

template <int V, bool U8>
__global__ void __launch_bounds__(256) sse_kernel(const JobDesc ref, const uint8_t *__restrict__ rec_u8,
                                                  int64_t rec_pitch, const float *__restrict__ rec_f32,
                                                  int64_t rec_pitch_f32, unsigned long long *acc_u64,
                                                  double *acc_f64) {
    constexpr int NW = V / 4 > 0 ? V / 4 : 1;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t h = (int64_t)ref.nbh * 8, w = (int64_t)ref.nbw * 8;
    unsigned long long su = 0;
    double sf = 0.0;
    for (int64_t y = warp; y < h; y += nwarps) {
        const uint8_t *a = ref.src + y * ref.src_pitch;
        for (int64_t x = (int64_t)lane * V; x < w; x += 32 * V) {
            uint32_t wa[NW];
            load_px<V>(a + x, wa);
            if constexpr (U8) {
                uint32_t wb[NW];
                load_px<V>(rec_u8 + y * rec_pitch + x, wb);
                if constexpr (V >= 8) {
                    unsigned aa = 0, bb = 0, ab = 0;  // at most 16 * 255^2 each
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        aa = __dp4a(wa[k], wa[k], aa);
                        bb = __dp4a(wb[k], wb[k], bb);
                        ab = __dp4a(wa[k], wb[k], ab);
                    }
                    su += (unsigned long long)aa + bb - 2ull * ab;
                } else {
                    const int d = (int)wa[0] - (int)wb[0];
                    su += (unsigned)(d * d);
                }
            } else {
                const float *b = rec_f32 + y * rec_pitch_f32 + x;
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const float d = b[k] - (float)((V >= 8) ? byte_of(wa[k >> 2], k & 3) : wa[0]);
                    s = __fmaf_rn(d, d, s);
                }
                sf += (double)s;
            }
        }
    }
    if constexpr (U8) {
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
    // launched as a programmatic dependent of the sweep kernel
    asm volatile("griddepcontrol.wait;" ::: "memory");
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
    forward_kernel<<<grid_for(nb, kFwdWarps * 32, 8), kFwdWarps * 32, 0, s>>>(job, Y);
    return cudaGetLastError();
}

cudaError_t launch_forward_f32(const JobDesc &job, int kind, float *Y, cudaStream_t s) {
    const int64_t nb = (int64_t)job.nbw * job.nbh;
    const DctConsts C = make_dct_consts();
    const ScaleConsts S = make_scale_consts();
    const int g = grid_for(nb, kFwdWarps * 32, 8);
    if (kind == RDCT_KIND_RDCT) forward_f32_kernel<RDCT_KIND_RDCT><<<g, kFwdWarps * 32, 0, s>>>(job, Y, C, S);
    else forward_f32_kernel<RDCT_KIND_DCT><<<g, kFwdWarps * 32, 0, s>>>(job, Y, C, S);
    return cudaGetLastError();
}

cudaError_t launch_compress(const int32_t *Y, int64_t nblocks, int32_t r, float *Yc, cudaStream_t s) {
    compress_kernel<<<grid_for(nblocks * r, 256, 16), 256, 0, s>>>(Y, nblocks, r, Yc, make_zigzag_table(),
                                                                   make_scale_consts());
    return cudaGetLastError();
}

template <int KIND>
static void launch_inverse_kind(int d, int g, const float *Yc, int64_t nbw, int64_t nbh, int32_t r, uint8_t *u8,
                                int64_t pitch, int u8_align, float *f32, int64_t pitch_f32, const ScaleConsts &S,
                                const DctConsts &C, cudaStream_t s) {
    switch (d) {
#define RDCT_ICASE(dd)                                                                                        \
    case dd:                                                                                                  \
        inverse_kernel<KIND, dd><<<g, 256, 0, s>>>(Yc, nbw, nbh, r, u8, pitch, u8_align, f32, pitch_f32, S, C); \
        break;
        RDCT_ICASE(0) RDCT_ICASE(1) RDCT_ICASE(2) RDCT_ICASE(3) RDCT_ICASE(4) RDCT_ICASE(5) RDCT_ICASE(6)
        RDCT_ICASE(7) RDCT_ICASE(8) RDCT_ICASE(9) RDCT_ICASE(10) RDCT_ICASE(11) RDCT_ICASE(12) RDCT_ICASE(13)
        RDCT_ICASE(14)
#undef RDCT_ICASE
        default: break;
    }
}

cudaError_t launch_inverse(const float *Yc, int64_t nbw, int64_t nbh, int32_t r, int kind, uint8_t *u8, int64_t pitch,
                           float *f32, int64_t pitch_f32, cudaStream_t s) {
    const int64_t nb = nbw * nbh;
    const int g = grid_for(nb, 256, 8);
    const int d = diag_class_host(r);
    const uintptr_t ua = reinterpret_cast<uintptr_t>(u8);
    const int u8_align = (ua % 8 == 0 && pitch % 8 == 0) ? 8 : 1;
    if (kind == RDCT_KIND_RDCT)
        launch_inverse_kind<RDCT_KIND_RDCT>(d, g, Yc, nbw, nbh, r, u8, pitch, u8_align, f32, pitch_f32,
                                            make_scale_consts(), DctConsts{}, s);
    else
        launch_inverse_kind<RDCT_KIND_DCT>(d, g, Yc, nbw, nbh, r, u8, pitch, u8_align, f32, pitch_f32, ScaleConsts{},
                                           make_dct_consts(), s);
    return cudaGetLastError();
}

cudaError_t launch_sse(const JobDesc &ref, const uint8_t *rec_u8, int64_t rec_pitch, const float *rec_f32,
                       int64_t rec_pitch_f32, unsigned long long *acc_u64, double *acc_f64, cudaStream_t s) {
    const int64_t rows = (int64_t)ref.nbh * 8, w = (int64_t)ref.nbw * 8;
    const int g = grid_for(rows * 32, 256, 8);
    const uintptr_t a = reinterpret_cast<uintptr_t>(ref.src);
    const uintptr_t b = rec_u8 ? reinterpret_cast<uintptr_t>(rec_u8) : reinterpret_cast<uintptr_t>(rec_f32);
    const int64_t bp = rec_u8 ? rec_pitch : rec_pitch_f32 * 4;
    auto aligned = [&](int k) { return a % k == 0 && ref.src_pitch % k == 0 && (!rec_u8 || (b % k == 0 && bp % k == 0)); };
    // a row is a multiple of 8 pixels; 16-pixel steps need a multiple of 16
    const int V = (aligned(16) && w % 16 == 0) ? 16 : (aligned(8) ? 8 : 1);
#define RDCT_SSE(v)                                                                                                \
    do {                                                                                                           \
        if (rec_u8) sse_kernel<v, true><<<g, 256, 0, s>>>(ref, rec_u8, rec_pitch, rec_f32, rec_pitch_f32, acc_u64,  \
                                                          acc_f64);                                                \
        else sse_kernel<v, false><<<g, 256, 0, s>>>(ref, rec_u8, rec_pitch, rec_f32, rec_pitch_f32, acc_u64, acc_f64); \
    } while (0)
    if (V == 16) RDCT_SSE(16);
    else if (V == 8) RDCT_SSE(8);
    else RDCT_SSE(1);
#undef RDCT_SSE
    return cudaGetLastError();
}

cudaError_t launch_mse_finalize(const unsigned long long *acc_u64, const double *acc_f64, int use_u64,
                                double nsamples, double *mse, double *psnr, cudaStream_t s) {
    mse_finalize_kernel<<<1, 32, 0, s>>>(acc_u64, acc_f64, use_u64, nsamples, mse, psnr);
    return cudaGetLastError();
}

cudaError_t launch_sse576_to_double(void *slots, int32_t n, cudaStream_t s, void *slots8) {
    if (n <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n + 255) / 256));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sse576_to_double_kernel, slots, slots8, n);
}

// 2-D byte copy by the SMs, for host memory that the device reaches through
// the host page tables (pageable memory), where the copy engines would need
// the driver's staging: rows strided over grid.y, each row's elements of VEC
// bytes strided over the threads of grid.x.
template <int VEC>
__global__ void copy2d_kernel(uint8_t *dst, int64_t dpitch, const uint8_t *src, int64_t spitch, int32_t w, int32_t h) {
    const int32_t per_row = w / VEC;
    for (int32_t y = blockIdx.y; y < h; y += gridDim.y) {
        const uint8_t *s = src + (int64_t)y * spitch;
        uint8_t *d = dst + (int64_t)y * dpitch;
        for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < per_row; x += gridDim.x * blockDim.x) {
            if constexpr (VEC == 16) reinterpret_cast<uint4 *>(d)[x] = reinterpret_cast<const uint4 *>(s)[x];
            else if constexpr (VEC == 8) reinterpret_cast<uint2 *>(d)[x] = reinterpret_cast<const uint2 *>(s)[x];
            else d[x] = s[x];
        }
    }
}

bool device_pageable_access(int device) {
    int pma = 0, host_tables = 0;
    if (cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return pma == 1 && host_tables == 1;
}

bool is_pageable_host(const void *p, int64_t bytes) {
    const void *ends[2] = {p, static_cast<const uint8_t *>(p) + (bytes > 0 ? bytes - 1 : 0)};
    for (const void *q : ends) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeUnregistered) return false;
    }
    return true;
}

cudaError_t launch_copy2d(void *dst, int64_t dpitch, const void *src, int64_t spitch, int32_t w, int32_t h,
                          cudaStream_t s) {
    if (w <= 0 || h <= 0) return cudaSuccess;
    auto aligned = [&](int a) {
        return reinterpret_cast<uintptr_t>(dst) % a == 0 && reinterpret_cast<uintptr_t>(src) % a == 0 &&
               dpitch % a == 0 && spitch % a == 0 && w % a == 0;
    };
    const int vec = aligned(16) ? 16 : aligned(8) ? 8 : 1;
    const int32_t per_row = w / vec;
    const int tx = per_row >= 256 ? 256 : ((per_row + 31) / 32) * 32;
    const int gx = (per_row + tx * 4 - 1) / (tx * 4);
    const int gy = h < 4096 ? h : 4096;
    const dim3 grid((unsigned)(gx < 1 ? 1 : gx), (unsigned)gy);
    auto *d = static_cast<uint8_t *>(dst);
    auto *sp = static_cast<const uint8_t *>(src);
    if (vec == 16) copy2d_kernel<16><<<grid, tx, 0, s>>>(d, dpitch, sp, spitch, w, h);
    else if (vec == 8) copy2d_kernel<8><<<grid, tx, 0, s>>>(d, dpitch, sp, spitch, w, h);
    else copy2d_kernel<1><<<grid, tx, 0, s>>>(d, dpitch, sp, spitch, w, h);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, int kind, double *out,
                         int32_t nplanes, int32_t ntiles, cudaStream_t s) {
    // RDCT: the per-block kernel over the chunks; the exact DCT: the tensor-core kernel over the tiles
    if (!sweep_is_tiled(kind)) {
        if (nchunks <= 0) return cudaSuccess;
        return launch_sweep2(jobs, chunks, nchunks, out, s);
    }
    if (ntiles <= 0) return cudaSuccess;
    return launch_sweep_dct_tc(jobs, nplanes, ntiles, out, s);
}

cudaError_t launch_sweep_finalize(double *out, int32_t nplanes, int kind, cudaStream_t s) {
    if (nplanes <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((nplanes + 3) / 4));
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sweep_finalize_kernel, out, nplanes, kind);
}

}  // namespace rdct
