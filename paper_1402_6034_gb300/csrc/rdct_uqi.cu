// rdct_uqi.cu -- the universal quality index (UQI) that Sec. 3 of Cintra &
// Bayer uses beside PSNR and MSE (its definition is in the work the paper
// cites, Wang & Bovik 2002).
//
// For every 8x8 window of the reference x and the reconstruction y, sliding
// by one pixel,
//   Q = [2 s_xy / (s_x^2 + s_y^2)] * [2 mx my / (mx^2 + my^2)]
// (sample means, unbiased variances and covariance; a factor whose
// denominator is zero counts as 1), and the index is the mean of Q over all
// windows.  With window sums Sx, Sy, Sxx, Syy, Sxy over N = 64 pixels the
// normalisations cancel:
//   2 s_xy / (s_x^2 + s_y^2) = 2 (N Sxy - Sx Sy) / (N (Sxx + Syy) - Sx^2 - Sy^2)
//   2 mx my / (mx^2 + my^2)   = 2 Sx Sy / (Sx^2 + Sy^2)
// so for an 8-bit reconstruction every sum is an exact integer.
//
// One thread per window; a CTA of 16 x 16 threads stages the 23 x 23 pixels
// its windows cover in shared memory.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "rdct_internal.h"

namespace rdct {
namespace {

constexpr int kWin = 8;
constexpr int kTile = 16;
constexpr int kSpan = kTile + kWin - 1;

template <bool U8>
__global__ void __launch_bounds__(kTile *kTile) uqi_kernel(const uint8_t *__restrict__ x, int64_t xpitch,
                                                           const uint8_t *__restrict__ yu, const float *__restrict__ yf,
                                                           int64_t ypitch, int32_t w, int32_t h, double *sum) {
    __shared__ uint8_t sx[kSpan][kSpan];
    __shared__ typename std::conditional<U8, uint8_t, float>::type sy[kSpan][kSpan];
    __shared__ double red[kTile * kTile / 32];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    for (int k = tid; k < kSpan * kSpan; k += kTile * kTile) {
        const int r = k / kSpan, c = k - r * kSpan;
        const int gy = y0 + r, gx = x0 + c;
        const bool in = gy < h && gx < w;
        sx[r][c] = in ? x[(int64_t)gy * xpitch + gx] : 0;
        if constexpr (U8) sy[r][c] = in ? yu[(int64_t)gy * ypitch + gx] : 0;
        else sy[r][c] = in ? yf[(int64_t)gy * ypitch + gx] : 0.0f;
    }
    __syncthreads();
    double q = 0.0;
    const int wx = x0 + threadIdx.x, wy = y0 + threadIdx.y;
    if (wx + kWin <= w && wy + kWin <= h) {
        constexpr double N = kWin * kWin;
        if constexpr (U8) {
            int Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
#pragma unroll
            for (int i = 0; i < kWin; ++i)
#pragma unroll
                for (int j = 0; j < kWin; ++j) {
                    const int a = sx[threadIdx.y + i][threadIdx.x + j], b = sy[threadIdx.y + i][threadIdx.x + j];
                    Sx += a;
                    Sy += b;
                    Sxx += a * a;
                    Syy += b * b;
                    Sxy += a * b;
                }
            const long long A = (long long)kWin * kWin * Sxy - (long long)Sx * Sy;
            const long long B = (long long)kWin * kWin * (Sxx + Syy) - (long long)Sx * Sx - (long long)Sy * Sy;
            const long long C = (long long)Sx * Sx + (long long)Sy * Sy;
            const double f1 = B == 0 ? 1.0 : 2.0 * (double)A / (double)B;
            const double f2 = C == 0 ? 1.0 : 2.0 * (double)Sx * (double)Sy / (double)C;
            q = f1 * f2;
        } else {
            double Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
#pragma unroll
            for (int i = 0; i < kWin; ++i)
#pragma unroll
                for (int j = 0; j < kWin; ++j) {
                    const double a = sx[threadIdx.y + i][threadIdx.x + j], b = sy[threadIdx.y + i][threadIdx.x + j];
                    Sx += a;
                    Sy += b;
                    Sxx += a * a;
                    Syy += b * b;
                    Sxy += a * b;
                }
            const double A = N * Sxy - Sx * Sy;
            const double B = N * (Sxx + Syy) - Sx * Sx - Sy * Sy;
            const double C = Sx * Sx + Sy * Sy;
            const double f1 = B == 0.0 ? 1.0 : 2.0 * A / B;
            const double f2 = C == 0.0 ? 1.0 : 2.0 * Sx * Sy / C;
            q = f1 * f2;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((tid & 31) == 0) red[tid >> 5] = q;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kTile * kTile / 32; ++k) t += red[k];
        if (t != 0.0) atomicAdd(sum, t);
    }
}

__global__ void scale_kernel(double *v, double factor) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *v *= factor;
}

}  // namespace
}  // namespace rdct

using namespace rdct;

extern "C" rdct_status rdct_uqi(const rdct_plane *ref, const rdct_out *rec, double *q, rdct_stream stream) {
    rdct_status st = validate_plane(ref, "rdct_uqi");
    if (st) return st;
    if (!rec || (!rec->u8 && !rec->f32) || !q) return set_error(RDCT_ERR_ARG, "rdct_uqi: null reconstruction or output");
    if (reinterpret_cast<uintptr_t>(q) % 8) return set_error(RDCT_ERR_ARG, "rdct_uqi: misaligned output");
    if (rec->u8 && rec->pitch < ref->w) return set_error(RDCT_ERR_SHAPE, "rdct_uqi: u8 pitch smaller than width");
    if (!rec->u8 && rec->pitch_f32 < ref->w) return set_error(RDCT_ERR_SHAPE, "rdct_uqi: f32 pitch smaller than width");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t w = ref->w, h = ref->h;
    const dim3 grid((w - kWin + kTile) / kTile, (h - kWin + kTile) / kTile), block(kTile, kTile);
    RDCT_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(double), s));
    if (rec->u8)
        uqi_kernel<true><<<grid, block, 0, s>>>(ref->ptr, ref->pitch, rec->u8, nullptr, rec->pitch, w, h, q);
    else
        uqi_kernel<false><<<grid, block, 0, s>>>(ref->ptr, ref->pitch, nullptr, rec->f32, rec->pitch_f32, w, h, q);
    RDCT_CUDA_TRY(cudaGetLastError());
    const double windows = (double)(w - kWin + 1) * (double)(h - kWin + 1);
    scale_kernel<<<1, 32, 0, s>>>(q, 1.0 / windows);
    RDCT_CUDA_TRY(cudaGetLastError());
    return RDCT_OK;
}
