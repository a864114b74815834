// rdct_blocks.cuh -- per-block device bodies and the fused kernels of the
// RDCT path (Sec. 3 of Cintra & Bayer), shared by the translation units that
// instantiate them.
//
// Mapping: one thread owns one 8x8 block; a warp owns a strip of 32
// horizontally adjacent blocks of one block row, so every row load of a warp
// is 256 contiguous bytes.  Kernels are persistent (grid-stride over strips).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "rdct_device.cuh"
#include "rdct_internal.h"

namespace rdct {

// ------------------------------------------------------------- utilities

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Eight rows of one 8x8 block: w[2i] holds pixels 0..3 of row i, w[2i+1] 4..7.
__device__ __forceinline__ void load_block(const uint8_t *p, int64_t pitch, int align, uint32_t w[16]) {
    if (align >= 8) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p + i * pitch));
            w[2 * i] = v.x;
            w[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint8_t *q = p + i * pitch;
            w[2 * i] = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) | ((uint32_t)q[3] << 24);
            w[2 * i + 1] = (uint32_t)q[4] | ((uint32_t)q[5] << 8) | ((uint32_t)q[6] << 16) | ((uint32_t)q[7] << 24);
        }
    }
}

__device__ __forceinline__ void store_row_u8(uint8_t *p, int align, uint32_t lo, uint32_t hi) {
    if (align >= 8) {
        __stcs(reinterpret_cast<uint2 *>(p), make_uint2(lo, hi));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            p[k] = (uint8_t)(lo >> (8 * k));
            p[4 + k] = (uint8_t)(hi >> (8 * k));
        }
    }
}

__device__ __forceinline__ void store_row_f32(float *p, const float v[8]) {
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
        __stcs(reinterpret_cast<float4 *>(p) + 1, make_float4(v[4], v[5], v[6], v[7]));
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = v[k];
    }
}

// Y = C0 A C0^T (int32) from the 16 packed words of a block: row pass, then
// column pass, each the 22-addition butterfly.
__device__ __forceinline__ void forward_c0(const uint32_t w[16], int Y[8][8]) {
    int R[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int x[8];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            x[n] = (int)byte_of(w[2 * i], n);
            x[n + 4] = (int)byte_of(w[2 * i + 1], n);
        }
        c0_forward(x, R[i]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int c[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = R[i][j];
        c0_forward(c, o);
#pragma unroll
        for (int i = 0; i < 8; ++i) Y[i][j] = o[i];
    }
}

// ------------------------------------------------- exact-DCT (FP32) helpers

__device__ __forceinline__ void dct_fwd8(const float x[8], float X[8], const DctConsts &C) {
    float a[4], b[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        a[n] = x[n] + x[7 - n];
        b[n] = x[n] - x[7 - n];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int n = 0; n < 4; ++n) acc = __fmaf_rn(C.c[k * 8 + n], (k & 1) ? b[n] : a[n], acc);
        X[k] = acc;
    }
}

template <unsigned M>
__device__ __forceinline__ void dct_inv8(const float X[8], float x[8], const DctConsts &C) {
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        float ev = 0.0f, od = 0.0f;
        static_for<0, 8>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            if constexpr ((M >> k) & 1u) {
                if constexpr (k & 1) od = __fmaf_rn(C.c[k * 8 + n], X[k], od);
                else ev = __fmaf_rn(C.c[k * 8 + n], X[k], ev);
            }
        });
        x[n] = ev + od;
        x[7 - n] = ev - od;
    }
}

__device__ __forceinline__ void forward_dct(const uint32_t w[16], float Y[8][8], float A[8][8], const DctConsts &C) {
    float R[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            A[i][n] = (float)byte_of(w[2 * i], n);
            A[i][n + 4] = (float)byte_of(w[2 * i + 1], n);
        }
        dct_fwd8(A[i], R[i], C);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = R[i][j];
        dct_fwd8(c, o, C);
#pragma unroll
        for (int i = 0; i < 8; ++i) Y[i][j] = o[i];
    }
}

// -------------------------------------------------------- fused block bodies

// RDCT, retained zone = every anti-diagonal < D plus the ranks < r of diagonal D.
// Returns 576 * SSE of the block (exact).  With OUT & 1, the 8-bit
// reconstruction goes to dst when dst is not nullptr, and with e8 its squared
// error against the block is added to s8 (sum a^2 - 2 sum q a + sum q^2 from
// byte dot products: exact).
template <int D, int OUT>
__device__ __forceinline__ unsigned long long fused_block_rdct(const uint32_t w[16], int r, uint8_t *dst,
                                                               int64_t dpitch, int dalign, float *dstf,
                                                               int64_t fpitch, bool e8, unsigned long long &s8) {
    unsigned sumsq = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) sumsq = __dp4a(w[k], w[k], sumsq);

    int Y[8][8];
    forward_c0(w, Y);

    long long kept = 0;
    float Z[8][8];
    static_for<0, 8>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<0, 8>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            if constexpr (i + j <= D) {
                int z = weight(i, j) * Y[i][j];
                if constexpr (i + j == D) {
                    if (zz_rank(i, j) >= r) z = 0;
                }
                kept += (long long)z * Y[i][j];
                Z[i][j] = (float)z;
            } else {
                Z[i][j] = 0.0f;
            }
        });
    });

    // inverse: U = C0^T Z (columns), then E = U C0 (rows); E = 576 * Xhat
    float U[8][8];
    static_for<0, 8>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        constexpr unsigned m = col_mask(D, j);
        if constexpr (m != 0u) {
            float in[8], out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) in[i] = Z[i][j];
            c0t_inverse<m>(in, out);
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = out[i];
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = 0.0f;
        }
    });
    constexpr unsigned rm = row_mask(D);
    unsigned qq = 0, qx = 0;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        float E[8];
        c0t_inverse<rm>(U[n], E);
        if constexpr (OUT & 1) {
            if (dst != nullptr || e8) {  // uniform: batch planes may have no uint8 output
                int q[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) q[m] = q_from_576(E[m]);
                const uint32_t lo = pack4_sat(q[0], q[1], q[2], q[3]), hi = pack4_sat(q[4], q[5], q[6], q[7]);
                if (e8) {
                    qq = __dp4a(lo, lo, __dp4a(hi, hi, qq));
                    qx = __dp4a(lo, w[2 * n], __dp4a(hi, w[2 * n + 1], qx));
                }
                if (dst != nullptr) store_row_u8(dst + n * dpitch, dalign, lo, hi);
            }
        }
        if constexpr (OUT & 2) {
            float v[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = E[m] * (1.0f / 576.0f);
            store_row_f32(dstf + n * fpitch, v);
        }
    }
    if constexpr (OUT & 1) {
        if (e8) s8 += (unsigned long long)(sumsq + qq - 2u * qx);
    }
    return 576ull * (unsigned long long)sumsq - (unsigned long long)kept;
}

// Exact DCT twin in FP32; returns the block's SSE (FP32 sum of 64 squares).
// 8-bit output and its squared error (e8, exact integers) as for the RDCT.
template <int D, int OUT>
__device__ __forceinline__ float fused_block_dct(const uint32_t w[16], int r, const DctConsts &C, uint8_t *dst,
                                                 int64_t dpitch, int dalign, float *dstf, int64_t fpitch, bool e8,
                                                 unsigned long long &s8) {
    float A[8][8], Y[8][8];
    forward_dct(w, Y, A, C);
    static_for<0, 8>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<0, 8>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            if constexpr (i + j == D) {
                if (zz_rank(i, j) >= r) Y[i][j] = 0.0f;
            } else if constexpr (i + j > D) {
                Y[i][j] = 0.0f;
            }
        });
    });
    float U[8][8];
    static_for<0, 8>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        constexpr unsigned m = col_mask(D, j);
        if constexpr (m != 0u) {
            float in[8], out[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) in[i] = Y[i][j];
            dct_inv8<m>(in, out, C);
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = out[i];
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = 0.0f;
        }
    });
    constexpr unsigned rm = row_mask(D);
    float sse = 0.0f;
    unsigned qq = 0, qx = 0;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        float X[8];
        dct_inv8<rm>(U[n], X, C);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const float e = X[m] - A[n][m];
            sse = __fmaf_rn(e, e, sse);
        }
        if constexpr (OUT & 1) {
            if (dst != nullptr || e8) {
                int q[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) q[m] = q_of(X[m]);
                const uint32_t lo = pack4_sat(q[0], q[1], q[2], q[3]), hi = pack4_sat(q[4], q[5], q[6], q[7]);
                if (e8) {
                    qq = __dp4a(lo, lo, __dp4a(hi, hi, qq));
                    qx = __dp4a(lo, w[2 * n], __dp4a(hi, w[2 * n + 1], qx));
                }
                if (dst != nullptr) store_row_u8(dst + n * dpitch, dalign, lo, hi);
            }
        }
        if constexpr (OUT & 2) store_row_f32(dstf + n * fpitch, X);
    }
    if constexpr (OUT & 1) {
        if (e8) {
            unsigned sumsq = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) sumsq = __dp4a(w[k], w[k], sumsq);
            s8 += (unsigned long long)(sumsq + qq - 2u * qx);
        }
    }
    return sse;
}

// ---------------------------------------------------------- fused kernels

// acc: the plane's 576 * SSE (uint64, kind RDCT) or SSE (double, kind DCT);
// acc8: the squared error of the 8-bit reconstruction (uint64) or nullptr.
template <int D, int OUT, int KIND>
__global__ void __launch_bounds__(256) fused_single_kernel(const JobDesc job, void *acc, unsigned long long *acc8,
                                                           const DctConsts C) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nitems = job.nbh * job.segs;
    const bool e8 = acc8 != nullptr;
    unsigned long long s576 = 0, s8 = 0;
    double sd = 0.0;
    for (int it = warp; it < nitems; it += nwarps) {
        const int by = it / job.segs;
        const int bx = (it - by * job.segs) * 32 + lane;
        if (bx < job.nbw) {
            uint32_t w[16];
            load_block(job.src + (int64_t)by * 8 * job.src_pitch + (int64_t)bx * 8, job.src_pitch, job.align, w);
            uint8_t *dst = (OUT & 1) && job.dst ? job.dst + (int64_t)by * 8 * job.dst_pitch + (int64_t)bx * 8 : nullptr;
            float *dstf = (OUT & 2) ? job.dstf + (int64_t)by * 8 * job.dstf_pitch + (int64_t)bx * 8 : nullptr;
            if constexpr (KIND == RDCT_KIND_RDCT) {
                s576 += fused_block_rdct<D, OUT>(w, job.r, dst, job.dst_pitch, job.dalign, dstf, job.dstf_pitch, e8,
                                                 s8);
            } else {
                sd += (double)fused_block_dct<D, OUT>(w, job.r, C, dst, job.dst_pitch, job.dalign, dstf,
                                                      job.dstf_pitch, e8, s8);
            }
        }
    }
    if constexpr (KIND == RDCT_KIND_RDCT) {
        s576 = warp_sum_u64(s576);
        if (lane == 0 && s576) atomicAdd(reinterpret_cast<unsigned long long *>(acc), s576);
    } else {
        sd = warp_sum_f64(sd);
        if (lane == 0 && sd != 0.0) atomicAdd(reinterpret_cast<double *>(acc), sd);
    }
    if (e8) {
        s8 = warp_sum_u64(s8);
        if (lane == 0 && s8) atomicAdd(acc8, s8);
    }
}

template <int D, int OUT>
__device__ __forceinline__ unsigned long long run_chunk_rdct(const JobDesc &job, const Chunk &ch, int lane, bool e8,
                                                             unsigned long long &s8) {
    unsigned long long s576 = 0;
    for (int it = ch.item0; it < ch.item0 + ch.nitems; ++it) {
        const int by = it / job.segs;
        const int bx = (it - by * job.segs) * 32 + lane;
        if (bx < job.nbw) {
            uint32_t w[16];
            load_block(job.src + (int64_t)by * 8 * job.src_pitch + (int64_t)bx * 8, job.src_pitch, job.align, w);
            uint8_t *dst = (OUT & 1) && job.dst ? job.dst + (int64_t)by * 8 * job.dst_pitch + (int64_t)bx * 8 : nullptr;
            s576 += fused_block_rdct<D, OUT>(w, job.r, dst, job.dst_pitch, job.dalign, nullptr, 0, e8, s8);
        }
    }
    return s576;
}

// Persistent kernel over a chunk table (uneven planes, per-plane r).  One
// instantiation covers the anti-diagonal classes DLO..DHI so that classes with
// very different register needs run in separate launches at their own
// occupancy.  acc8: per-image squared error of the 8-bit reconstruction, or
// nullptr.
template <int OUT, int DLO, int DHI>
__global__ void __launch_bounds__(256) fused_batch_kernel(const JobDesc *__restrict__ jobs,
                                                          const Chunk *__restrict__ chunks, int nchunks,
                                                          unsigned long long *acc, unsigned long long *acc8) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const bool e8 = acc8 != nullptr;
    for (int c = warp; c < nchunks; c += nwarps) {
        const Chunk ch = chunks[c];
        const JobDesc job = jobs[ch.job];
        unsigned long long s = 0, s8 = 0;
        static_for<DLO, DHI + 1>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            if (ch.cls == d) s = run_chunk_rdct<d, OUT>(job, ch, lane, e8, s8);
        });
        s = warp_sum_u64(s);
        if (lane == 0 && s) atomicAdd(&acc[job.image], s);
        if (e8) {
            s8 = warp_sum_u64(s8);
            if (lane == 0 && s8) atomicAdd(&acc8[job.image], s8);
        }
    }
}

// Resident CTAs per SM of `kernel` at `threads` threads (occupancy limit).
template <typename K>
inline int resident_ctas(K kernel, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

// Launch a persistent kernel over `units` warp work units with grid =
// min(units / warps, SMs x resident CTAs), at most ctas_per_sm CTAs per SM
// when ctas_per_sm > 0.
template <typename K, typename... Args>
inline void launch_persistent(K kernel, int64_t units, int ctas_per_sm, int warps, cudaStream_t s, Args... args) {
    const int threads = warps * 32;
    int per_sm = resident_ctas(kernel, threads);
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t g = (int64_t)sm_count() * per_sm;
    const int64_t need = (units + warps - 1) / warps;
    if (g > need) g = need;
    kernel<<<(int)(g < 1 ? 1 : g), threads, 0, s>>>(args...);
}

// Persistent launch of a kernel that stages rows through a shared-memory
// ring: at most max_ctas CTAs per SM, and the shared-memory carve-out set to
// the smallest size that holds them, so the rest of the SM's 256 KB stays L1
// (the copies into the ring are cached in L1; a larger carve-out measurably
// slows them down).
// overlap: launch as a programmatic dependent of the previous kernel in the
// stream (the kernel must trigger and wait with griddepcontrol itself).
template <typename K, typename... Args>
inline cudaError_t launch_staged(K kernel, int64_t units, int ctas_per_sm, int warps, int max_ctas, int smem_per_cta,
                                 bool overlap, cudaStream_t s, Args... args) {
    const int threads = warps * 32;
    int per_sm = resident_ctas(kernel, threads);
    if (per_sm > max_ctas) per_sm = max_ctas;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const int pct = (int)((100LL * per_sm * (smem_per_cta + 1024) + 228 * 1024 - 1) / (228 * 1024));
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
    int64_t g = (int64_t)sm_count() * per_sm;
    const int64_t need = (units + warps - 1) / warps;
    if (g > need) g = need;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g < 1 ? 1 : g));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = overlap ? attr : nullptr;
    cfg.numAttrs = overlap ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Single-plane fused launch for one output mode and transform kind; the
// anti-diagonal class d selects the specialised kernel.
template <int OUT, int KIND>
cudaError_t launch_single_variant(int d, int64_t items, int ctas_per_sm, int warps, const JobDesc &job, void *acc,
                                  unsigned long long *acc8, const DctConsts &C, cudaStream_t s);

}  // namespace rdct
