// rdct_sweep2.cuh -- the r sweep of Sec. 3 in one pass per plane.
//
// The transforms are orthogonal (Sec. 2), so the squared error of the
// reconstruction that keeps the first r zigzag coefficients is the energy of
// the dropped orthonormal coefficients (Parseval).  One pass per plane
// therefore gives the error for every r: each thread transforms its blocks,
// adds every coefficient's energy into 64 per-position bins held in
// registers, and once per chunk the warp reduces the bins and adds them to the
// plane's 64 zigzag-ordered bins; suffix sums then give SSE(r), r = 1..64.
//
// RDCT: Y = C0 A C0^T exactly (dp4a row pass on packed pixels, int32 column
// butterfly); the orthonormal energy of Y_ij is W_ij Y_ij^2 / 576, so the bins
// hold integer Y^2 sums (exact) and the weights are applied at the flush.
// DCT: C A C^T in FP32 (even/odd split, FMAs with the cos constants, on
// f32x2 pairs of rows and then of columns), FP32 bins, FP64 plane bins.
// Staging, strip cursors and chunking are those of the fused kernel.
#pragma once
#include "rdct_fused2.cuh"

namespace rdct {

// The DC energy is never needed (every r keeps the DC coefficient), so the
// bins hold AC energies only.  Every AC row of C0 sums to zero, so an AC
// coefficient is sum k a with sum k = 0 and entries of k in {-1, 0, 1}, at
// most 32 of them +1: |Y_ij| <= 32 * 255 = 8160 and Y^2 < 2^26.  A thread
// adds kFusedVRows blocks per strip and kSweepChunkStrips strips per chunk,
// and flushes its 32-bit bins at the latest after kSweepFlushChunks chunks:
constexpr int kSweepFlushChunks = 4;
static_assert(kSweepFlushChunks * kSweepChunkStrips * kFusedVRows * 8160ull * 8160ull < (1ull << 32),
              "sweep bins overflow");
// (the largest AC coefficient, for the bound above)
__host__ __device__ constexpr int max_ac_coefficient() {
    int m = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            if (i == 0 && j == 0) continue;
            int pos = 0;
            for (int y = 0; y < 8; ++y)
                for (int x = 0; x < 8; ++x) pos += c0_entry(i, y) * c0_entry(j, x) > 0 ? 1 : 0;
            m = pos > m ? pos : m;
        }
    return 255 * m;
}
static_assert(max_ac_coefficient() <= 8160, "AC coefficient bound");
// zigzag rank of bin p = 8 i + j (for the flush's per-lane atomics)
struct ZzRanks {
    unsigned char r[64];
};
constexpr ZzRanks make_zz_ranks() {
    ZzRanks t{};
    for (int p = 0; p < 64; ++p) t.r[p] = (unsigned char)zz_rank(p >> 3, p & 7);
    return t;
}
__constant__ ZzRanks kSweepZz = make_zz_ranks();

// One output column at a time: column j of C0 A (the row pass, two dp4a per
// row on the packed pixels), then the column butterfly, then its eight
// energies; only eight intermediates are live next to the 64 bins.
__device__ __forceinline__ void sweep_rdct_block(const uint2 (&w)[8], unsigned (&bins)[64]) {
    static_for<0, 8>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        int c[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            c[i] = dp4a_us_imm<c0_row_word(j, 0)>(w[i].x, dp4a_us_imm<c0_row_word(j, 1)>(w[i].y, 0));
        c0_forward(c, o);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i + j > 0) bins[i * 8 + j] += (unsigned)(o[i] * o[i]);
    });
}

// The constants of the factored 8-point DCT as f32x2 pairs (c, c), built once
// per thread and kept in registers: s = C[0][0] = C[4][0] (sqrt(1/8)),
// c_m = C[1][.] and C[2][.] entries = cos(m pi / 16) / 2, and the negatives
// the odd rows need.
struct DctPairs {
    f2 s, c2, c6, nc2, c1, c3, c5, c7, nc1, nc5, nc7;
};
__device__ __forceinline__ DctPairs dct_pairs(const DctConsts &C) {
    auto p = [](float v) { return f2_make(v, v); };
    DctPairs d;
    d.s = p(C.c[0]);
    d.c2 = p(C.c[16]);
    d.c6 = p(C.c[17]);
    d.nc2 = p(-C.c[16]);
    d.c1 = p(C.c[8]);
    d.c3 = p(C.c[9]);
    d.c5 = p(C.c[10]);
    d.c7 = p(C.c[11]);
    d.nc1 = p(-C.c[8]);
    d.nc5 = p(-C.c[10]);
    d.nc7 = p(-C.c[11]);
    return d;
}

// 8-point orthonormal DCT of an f32x2 pair of vectors, factored by the
// symmetries of C (rows 2k even about the centre, rows 2k+1 odd, and rows 0,
// 4, 2, 6 again even / odd on the half sums): 36 f32x2 operations with 11
// constant pairs held in registers.
__device__ __forceinline__ void dct8_f2_factored(const f2 (&x)[8], f2 (&X)[8], const DctPairs &K) {
    f2 a[4], b[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        a[n] = x[n] + x[7 - n];
        b[n] = x[n] - x[7 - n];
    }
    const f2 e03 = a[0] + a[3], e12 = a[1] + a[2], d03 = a[0] - a[3], d12 = a[1] - a[2];
    X[0] = mul2(K.s, e03 + e12);
    X[4] = mul2(K.s, e03 - e12);
    X[2] = fma2(K.c2, d03, mul2(K.c6, d12));
    X[6] = fma2(K.c6, d03, mul2(K.nc2, d12));
    X[1] = fma2(K.c7, b[3], fma2(K.c5, b[2], fma2(K.c3, b[1], mul2(K.c1, b[0]))));
    X[3] = fma2(K.nc5, b[3], fma2(K.nc1, b[2], fma2(K.nc7, b[1], mul2(K.c3, b[0]))));
    X[5] = fma2(K.c3, b[3], fma2(K.c7, b[2], fma2(K.nc1, b[1], mul2(K.c5, b[0]))));
    X[7] = fma2(K.nc1, b[3], fma2(K.c3, b[2], fma2(K.nc5, b[1], mul2(K.c7, b[0]))));
}

// Exact DCT energies of one block with f32x2 arithmetic: the row pass runs on
// pairs of rows, the column pass on pairs of columns.  Pixels become floats
// by placing each byte under the exponent of 2^23 (a byte permute) and
// subtracting 2^23, exactly.
__device__ __forceinline__ void sweep_dct_block(const uint2 (&w)[8], float (&bins)[64], const DctPairs &C) {
    const f2 two23 = f2_make(8388608.0f, 8388608.0f);
    float R[8][8];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        f2 x[8], X[8];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const unsigned sel = 0x7540u + (unsigned)n;
            x[n] = f2_make(__int_as_float((int)__byte_perm(w[i].x, 0x4B000000u, sel)),
                           __int_as_float((int)__byte_perm(w[i + 1].x, 0x4B000000u, sel))) - two23;
            x[n + 4] = f2_make(__int_as_float((int)__byte_perm(w[i].y, 0x4B000000u, sel)),
                               __int_as_float((int)__byte_perm(w[i + 1].y, 0x4B000000u, sel))) - two23;
        }
        dct8_f2_factored(x, X, C);
#pragma unroll
        for (int k = 0; k < 8; ++k) f2_split(X[k], R[i][k], R[i + 1][k]);
    }
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        f2 c[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = f2_make(R[i][j], R[i][j + 1]);
        dct8_f2_factored(c, o, C);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float y0, y1;
            f2_split(o[i], y0, y1);
            if (i + j > 0) bins[i * 8 + j] = __fmaf_rn(y0, y0, bins[i * 8 + j]);
            bins[i * 8 + j + 1] = __fmaf_rn(y1, y1, bins[i * 8 + j + 1]);
        }
    }
}

// Sum of a 32-bit value over the warp in 64 bits (two 16-bit halves, each
// summed with one warp reduction).
__device__ __forceinline__ unsigned long long warp_sum_u32_wide(unsigned v) {
    const unsigned lo = __reduce_add_sync(0xffffffffu, v & 0xFFFFu);
    const unsigned hi = __reduce_add_sync(0xffffffffu, v >> 16);
    return ((unsigned long long)hi << 16) + lo;
}

// The warp's 63 AC bins into the plane's zigzag bins: each bin summed over the
// warp, lane l keeping the totals of bins l and 32 + l, then two atomics per
// lane.
template <int KIND>
__device__ __forceinline__ void sweep_flush(double *plane_bins, unsigned (&ub)[64], float (&fb)[64], int lane) {
    unsigned long long u0 = 0ull, u1 = 0ull;
    float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
    for (int p = 1; p < 64; ++p) {
        if constexpr (KIND == RDCT_KIND_RDCT) {
            const unsigned long long s = warp_sum_u32_wide(ub[p]) * (unsigned)weight(p >> 3, p & 7);
            if (lane == (p & 31)) {
                if (p < 32) u0 = s;
                else u1 = s;
            }
            ub[p] = 0u;
        } else {
            const float s = warp_sum_f32(fb[p]);
            if (lane == (p & 31)) {
                if (p < 32) f0 = s;
                else f1 = s;
            }
            fb[p] = 0.0f;
        }
    }
    const int k0 = kSweepZz.r[lane], k1 = kSweepZz.r[32 + lane];
    if constexpr (KIND == RDCT_KIND_RDCT) {
        unsigned long long *b = reinterpret_cast<unsigned long long *>(plane_bins);
        if (u0) atomicAdd(b + k0, u0);
        if (u1) atomicAdd(b + k1, u1);
    } else {
        if (f0 != 0.0f) atomicAdd(plane_bins + k0, (double)f0);
        if (f1 != 0.0f) atomicAdd(plane_bins + k1, (double)f1);
    }
}

// Persistent sweep kernel over a chunk table (job = plane; out = [planes][64]
// zigzag-ordered bins: uint64 576-scaled energies for RDCT, double for DCT;
// the DC bin stays 0).  Each warp takes a contiguous run of chunks, so that
// consecutive chunks mostly belong to one plane and the bins are flushed only
// when the plane changes or after kSweepFlushChunks chunks.
template <int KIND>
__global__ void __launch_bounds__(128, KIND == RDCT_KIND_RDCT ? 4 : 3) sweep2_kernel(const Fused2Args args,
                                                                                   double *out, const DctConsts C) {
    constexpr int THREADS = 128;
    __shared__ uint2 ring[kStages * 8 * kVRows * THREADS];
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    // this warp's chunks [c0, c1): the cursors step by one chunk and stop at c1
    Fused2Args a = args;
    const int gw = (int)((int64_t)warp * args.nchunks / nwarps);
    a.nchunks = (int)((int64_t)(warp + 1) * args.nchunks / nwarps);
    // launched as a programmatic dependent of the table builder (which also clears the bins)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    unsigned ub[64];
    float fb[64];
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        ub[p] = 0u;
        fb[p] = 0.0f;
    }
    const DctPairs K = dct_pairs(C);
    Cursor fc{gw, 0, 0, 0, 0, 0};
    cursor_load<false>(a, fc, lane);
    Cursor cc = fc;
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (fc.c < a.nchunks) {
            fetch_strip<THREADS>(a.jobs[fc.job], fc.rp, fc.bx, ring, s);
            cursor_next<false>(a, fc, 1, lane);
        } else {
            cp_async_commit();
        }
    }
    int stage = 0, since_flush = 0;
    while (cc.c < a.nchunks) {
        cp_async_wait<kStages - 2>();
        const JobDesc &job = a.jobs[cc.job];
        const int by = cc.rp * kVRows;
        const int nblk = by < job.nbh ? (job.nbh - by >= kVRows ? kVRows : job.nbh - by) : 0;
        const int refill = stage == 0 ? kStages - 1 : stage - 1;
        if (fc.c < a.nchunks) {
            fetch_strip<THREADS>(a.jobs[fc.job], fc.rp, fc.bx, ring, refill);
            cursor_next<false>(a, fc, 1, lane);
        } else {
            cp_async_commit();
        }
        // RDCT: both blocks unrolled so that their work interleaves; DCT: one
        // after the other (its FP32 intermediates leave no registers to spare)
#pragma unroll (KIND == RDCT_KIND_RDCT ? kVRows : 1)
        for (int v = 0; v < kVRows; ++v) {
            if (v < nblk) {
                uint2 w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w[i] = ring[((stage * kVRows + v) * 8 + i) * THREADS + threadIdx.x];
                if constexpr (KIND == RDCT_KIND_RDCT) sweep_rdct_block(w, ub);
                else sweep_dct_block(w, fb, K);
            }
        }
        stage = stage + 1 == kStages ? 0 : stage + 1;
        const int plane = cc.job;
        const int cprev = cc.c;
        cursor_next<false>(a, cc, 1, lane);
        if (cc.c != cprev) {
            if (++since_flush == kSweepFlushChunks || cc.c >= a.nchunks || cc.job != plane) {
                sweep_flush<KIND>(out + (int64_t)plane * 64, ub, fb, lane);
                since_flush = 0;
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace rdct
