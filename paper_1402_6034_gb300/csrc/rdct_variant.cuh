// rdct_variant.cuh -- the block experiment of Sec. 3 for the other transforms
// the paper names: the signed DCT it compares against, and the floor / ceiling
// generalisations of C0 = [2C] that its conclusion proposes (Sec. 4).
//
// Unlike C0, these matrices have no diagonal Gram matrix (sign(C), ceil(2C))
// or need a full orthogonaliser, so the scaling cannot be folded into integer
// weights.  Each block A goes to Y = F A F^T, keeps the first r zigzag
// coefficients and is rebuilt as X = G Yhat G^T, with F and G dense FP32
// matrices passed by value (kernel parameters: constant-bank operands).
//
// One thread per 8x8 block.  The anti-diagonal class D of r is a template
// parameter, so only the rows and columns that can hold kept coefficients
// are computed: the forward row pass produces columns j <= D only, the
// column pass the kept zone i + j <= D only, and the inverse reads that zone.
#pragma once

#include "rdct_blocks.cuh"

namespace rdct {

// Pixel n (0..3) of a packed word as an exact float without a conversion
// instruction: the byte goes under the exponent of 2^23 (one byte permute)
// and 2^23 is subtracted (one add), both on full-rate pipes.
__device__ __forceinline__ float px_float(uint32_t w, int n) {
    return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7540u + (unsigned)n)) - 8388608.0f;
}

template <int D>
__device__ __forceinline__ float variant_block(const uint32_t w[16], int r, const MatConsts &M, uint8_t *dst,
                                               int64_t dpitch, int dalign, float *dstf, int64_t fpitch) {
    constexpr int K = D < 7 ? D + 1 : 8;  // columns (and rows) of Y that can be kept
    // Row pass: R[i][k] = sum_n A[i][n] F[k][n] for k < K.
    float R[8][K];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float a[8];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            a[n] = px_float(w[2 * i], n);
            a[n + 4] = px_float(w[2 * i + 1], n);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float acc = 0.0f;
#pragma unroll
            for (int n = 0; n < 8; ++n) acc = __fmaf_rn(M.f[k * 8 + n], a[n], acc);
            R[i][k] = acc;
        }
    }
    // Column pass on the kept zone, column by column so that each column of R
    // dies once used: Y[i][j] = sum_n F[i][n] R[n][j], i + j <= D.
    float Y[K][K];
    static_for<0, K>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        static_for<0, K>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if constexpr (i + j <= D) {
                float acc = 0.0f;
#pragma unroll
                for (int n = 0; n < 8; ++n) acc = __fmaf_rn(M.f[i * 8 + n], R[n][j], acc);
                if constexpr (i + j == D) {
                    if (zz_rank(i, j) >= r) acc = 0.0f;
                }
                Y[i][j] = acc;
            }
        });
    });
    // Inverse, one output row n at a time with only the kept zone live:
    // V[j] = sum_i G[n][i] Yhat[i][j], then X[n][m] = sum_j V[j] G[m][j].
    float sse = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        float V[K];
        static_for<0, K>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            float acc = 0.0f;
            static_for<0, K>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if constexpr (i + j <= D) acc = __fmaf_rn(M.g[n * 8 + i], Y[i][j], acc);
            });
            V[j] = acc;
        });
        float X[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < K; ++j) acc = __fmaf_rn(M.g[m * 8 + j], V[j], acc);
            X[m] = acc;
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const float e = X[m] - px_float(w[2 * n + (m >> 2)], m & 3);
            sse = __fmaf_rn(e, e, sse);
        }
        if (dst != nullptr) {
            int q[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) q[m] = q_of(X[m]);
            store_row_u8(dst + n * dpitch, dalign, pack4_sat(q[0], q[1], q[2], q[3]),
                         pack4_sat(q[4], q[5], q[6], q[7]));
        }
        if (dstf != nullptr) store_row_f32(dstf + n * fpitch, X);
    }
    return sse;
}

// Warps take block-row segments of 32 blocks (one block per lane); the plane's
// squared error is summed per thread in FP64 and added once per warp.  Launch
// bounds: four CTAs per SM (128 registers) while the class fits without
// spills (anti-diagonal class up to 3, r <= 10), three up to class 6, two
// above.
template <int D>
__global__ void __launch_bounds__(128, D <= 3 ? 4 : D <= 6 ? 3 : 2) variant_kernel(const JobDesc job, const MatConsts M, double *acc) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nitems = job.nbh * job.segs;
    double s = 0.0;
    for (int it = warp; it < nitems; it += nwarps) {
        const int by = it / job.segs;
        const int bx = (it - by * job.segs) * 32 + lane;
        if (bx < job.nbw) {
            uint32_t w[16];
            load_block(job.src + (int64_t)by * 8 * job.src_pitch + (int64_t)bx * 8, job.src_pitch, job.align, w);
            uint8_t *dst = job.dst ? job.dst + (int64_t)by * 8 * job.dst_pitch + (int64_t)bx * 8 : nullptr;
            float *dstf = job.dstf ? job.dstf + (int64_t)by * 8 * job.dstf_pitch + (int64_t)bx * 8 : nullptr;
            s += (double)variant_block<D>(w, job.r, M, dst, job.dst_pitch, job.dalign, dstf, job.dstf_pitch);
        }
    }
    s = warp_sum_f64(s);
    if (lane == 0 && s != 0.0) atomicAdd(acc, s);
}

template <int D>
cudaError_t launch_variant_d(const JobDesc &job, const MatConsts &M, double *acc, cudaStream_t s) {
    launch_persistent(variant_kernel<D>, (int64_t)job.nbh * job.segs, 0, 4, s, job, M, acc);
    return cudaGetLastError();
}

}  // namespace rdct
