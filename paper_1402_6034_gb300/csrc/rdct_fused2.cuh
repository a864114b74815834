// rdct_fused2.cuh -- the fused RDCT kernel (Sec. 3 of Cintra & Bayer: forward
// transform, zonal truncation with the S scaling of Sec. 2, inverse, squared
// error) shaped for sm_103a issue rates.
//
// Per 8x8 block (a thread owns two vertically adjacent blocks, a and b):
//   * rows of pixels arrive through a per-thread cp.async ring in shared
//     memory (double-buffered, no block barriers: each thread only
//     reads what it copied itself);
//   * row pass: every output of C0 applied to a row is one pair of byte dot
//     products (dp4a) of the packed pixels with a row of C0 as signed bytes,
//     so pixels are never unpacked;
//   * column pass: the 22-addition C0 butterfly in int32; the compiler drops
//     every output that r never keeps;
//   * compression: kept coefficients become Z = W Y with W = 576 d_i^2 d_j^2,
//     converted exactly to FP32 in units of 2^-149 (subnormal range);
//   * inverse: C0^T butterflies in FP32, exact because every value is an
//     integer multiple of 2^-149 below 2^24 units; every value from here on is
//     an f32x2 pair (block a, block b), so one instruction serves both blocks;
//   * output: one f32x2 multiply by 1/576 leaves round(Xhat) in the bit
//     pattern of each float (negative values carry the sign bit), and
//     cvt.pack.sat clamps to [0, 255] and packs four pixels per two
//     instructions;
//   * error: 576 SSE = 576 sum x^2 - sum_kept W Y^2 (Parseval, the transform
//     is orthogonal), with sum x^2 from dp4a and the kept energies summed
//     per weight group in 32 bits: exact;
//   * from r = 36 the same integers come from the coefficients that are
//     dropped instead (576 Xhat = 576 A - C0^T (W o Y_dropped) C0 and
//     576 SSE = sum_dropped W Y^2), so the work shrinks as r approaches 64,
//     where the reconstruction is the block itself;
//   * optionally the squared error of the 8-bit reconstruction, from byte dot
//     products of the packed output with itself and with the pixels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "rdct_blocks.cuh"

namespace rdct {

// ------------------------------------------------------------ f32x2 pairs

struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_make(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_split(f2 r, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r.v));
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 operator-(f2 a) { return f2{0ull} - a; }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}

// ------------------------------------------------------------ int helpers

// a (four unsigned bytes) . b (four signed bytes) + c
__device__ __forceinline__ int dp4a_us(unsigned a, unsigned b, int c) {
    int d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// The same with b a compile-time constant, given to the instruction as an
// immediate operand (no register has to hold it).
template <unsigned B>
__device__ __forceinline__ int dp4a_us_imm(unsigned a, int c) {
    int d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "n"(B), "r"(c));
    return d;
}
// Weight group of W_ij (six distinct values).
__host__ __device__ constexpr int weight_group(int i, int j) {
    const int w = weight(i, j);
    return w == 9 ? 0 : w == 12 ? 1 : w == 16 ? 2 : w == 18 ? 3 : w == 24 ? 4 : 5;
}
__host__ __device__ constexpr int group_weight(int g) {
    return g == 0 ? 9 : g == 1 ? 12 : g == 2 ? 16 : g == 3 ? 18 : g == 4 ? 24 : 36;
}

// --------------------------------------------------------------- block body

// Rows i holding retained coefficients in column j, and columns holding any,
// when exactly the first R zigzag coefficients are kept.
__host__ __device__ constexpr unsigned kept_col_mask(int R, int j) {
    unsigned m = 0u;
    for (int i = 0; i < 8; ++i)
        if (zz_rank(i, j) < R) m |= 1u << i;
    return m;
}
__host__ __device__ constexpr unsigned kept_row_mask(int R) {
    unsigned m = 0u;
    for (int j = 0; j < 8; ++j)
        if (kept_col_mask(R, j) != 0u) m |= 1u << j;
    return m;
}
// The same for the coefficients that are dropped (zigzag rank >= R).
__host__ __device__ constexpr unsigned drop_col_mask(int R, int j) {
    return ~kept_col_mask(R, j) & 0xFFu;
}
__host__ __device__ constexpr unsigned drop_row_mask(int R) {
    unsigned m = 0u;
    for (int j = 0; j < 8; ++j)
        if (drop_col_mask(R, j) != 0u) m |= 1u << j;
    return m;
}

// Where the reconstruction is built from the coefficients that are dropped
// rather than from those that are kept.  With every coefficient kept the
// scaled inverse returns the block exactly (C0^T (W o Y) C0 = 576 A, since
// C0^T diag(g)^-1 C0 = I for C0 C0^T = diag(g), Sec. 2), so
//   576 Xhat = 576 A - C0^T (W o Y_dropped) C0,
//   576 SSE  = sum over the dropped positions of W Y^2   (Parseval),
// the same integers as the kept form, in work that shrinks with 64 - r.
// Measured on a 600-frame 4K clip (fraction of HBM, kept / dropped form):
// r = 33 0.713 / 0.672, r = 35 0.712 / 0.701, r = 36 0.697 / 0.729,
// r = 40 0.685 / 0.798, r = 44 0.650 / 0.815; so the dropped form from r = 36.
__host__ __device__ constexpr bool drop_form(int R) { return R > 35; }

// Y = C0 A C0^T of one block: every output of the row pass is a pair of byte
// dot products of the packed pixels with a row of C0 as signed bytes (dp4a),
// the column pass the 22-addition butterfly in int32.
__device__ __forceinline__ void forward_c0_int(const uint2 (&w)[8], int (&Y)[8][8]) {
    int R[8][8];
    static_for<0, 8>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            R[i][k] = dp4a_us_imm<c0_row_word(k, 0)>(w[i].x, dp4a_us_imm<c0_row_word(k, 1)>(w[i].y, 0));
    });
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

// The forward transform of both blocks of a column pair at once, on packed
// pairs of 16-bit lanes (block a low, block b high): an addition or
// subtraction of two 32-bit words is exact in each lane as long as every true
// lane value stays within [-32768, 32767] (a carry or borrow out of the low
// lane is absorbed when the lanes are read back: lo = the sign-extended low
// half, hi = (word + 2^15) >> 16).  Every value on the path is at most
// 8 * 2040 = 16320 in magnitude, so the 22-addition butterflies of the row and
// the column pass serve both blocks with one integer addition each, on the
// integer ALU, instead of byte dot products on the multiply pipe.  The
// compiler drops every output (and lane read) that the zone in use never needs.
__device__ __forceinline__ void forward_pair16(const uint2 (&wa)[8], const uint2 (&wb)[8], int (&Ya)[8][8],
                                               int (&Yb)[8][8]) {
    unsigned R[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        unsigned x[8];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            // byte n of each block's word into the low byte of its lane
            const unsigned sel = (unsigned)n * 0x11u + (unsigned)(4 + n) * 0x1100u;
            x[n] = __byte_perm(wa[i].x, wb[i].x, sel) & 0x00FF00FFu;
            x[n + 4] = __byte_perm(wa[i].y, wb[i].y, sel) & 0x00FF00FFu;
        }
        c0_forward(x, R[i]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        unsigned c[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = R[i][j];
        c0_forward(c, o);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            Ya[i][j] = (int)(int16_t)(o[i] & 0xFFFFu);
            Yb[i][j] = ((int)o[i] + 0x8000) >> 16;
        }
    }
}

// Which form of the forward transform a kernel for exactly R kept
// coefficients uses: the packed 16-bit lanes move the work from the multiply
// pipe (dp4a) to the integer ALU, which pays where the multiply pipe is the
// busier one.  Measured on a 600-frame 4K clip, packed against dp4a: +1 to
// +2% at r = 16..23, +1 to +3.5% at r = 29..34, +1 to +2% at r = 55..58;
// within 0.5% at r = 6..12 and 24; 3 to 7% slower at r = 36..53 (there the
// reconstruction from the dropped coefficients already loads the ALU).
__host__ __device__ constexpr bool packed_forward(int R) {
    return (R >= 16 && R <= 24) || (R >= 28 && R <= 34) || (R >= 55 && R <= 58);
}

template <int R>
__device__ __forceinline__ void forward_pair(const uint2 (&wa)[8], const uint2 (&wb)[8], int (&Ya)[8][8],
                                             int (&Yb)[8][8]) {
    if constexpr (packed_forward(R)) {
        forward_pair16(wa, wb, Ya, Yb);
    } else {
        forward_c0_int(wa, Ya);
        forward_c0_int(wb, Yb);
    }
}

// Sum of squared pixels of both blocks (byte dot products).
__device__ __forceinline__ unsigned pair_sumsq(const uint2 (&wa)[8], const uint2 (&wb)[8]) {
    unsigned s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        s = __dp4a(wa[i].x, wa[i].x, s);
        s = __dp4a(wa[i].y, wa[i].y, s);
        s = __dp4a(wb[i].x, wb[i].x, s);
        s = __dp4a(wb[i].y, wb[i].y, s);
    }
    return s;
}

// Output of row n of both blocks from E = 576 Xhat (f32x2 pairs in units of
// 2^-149): one f32x2 multiply by fl(1/576) leaves round(Xhat) in the bit
// pattern, cvt.pack.sat clamps and packs.  The packed bytes q are stored
// (dst may be nullptr: error only) and, with E8, their squared error against
// the pixels is gathered as sum q^2 and sum q a (byte dot products), so that
// sum (q - a)^2 = sum a^2 - 2 sum q a + sum q^2 is exact.
template <bool SMEM, bool E8>
__device__ __forceinline__ void emit_row(const f2 (&E)[8], int n, const uint2 &pa, const uint2 &pb, uint8_t *dst,
                                         int64_t dpitch, int dalign, bool has_b, unsigned &qq, unsigned &qx) {
    const f2 inv576 = f2_make(1.0f / 576.0f, 1.0f / 576.0f);
    int qa[8], qb[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        float x, y;
        f2_split(mul2(E[m], inv576), x, y);
        qa[m] = __float_as_int(x);
        qb[m] = __float_as_int(y);
    }
    const uint32_t a0 = pack4_sat(qa[0], qa[1], qa[2], qa[3]), a1 = pack4_sat(qa[4], qa[5], qa[6], qa[7]);
    const uint32_t b0 = pack4_sat(qb[0], qb[1], qb[2], qb[3]), b1 = pack4_sat(qb[4], qb[5], qb[6], qb[7]);
    if constexpr (E8) {
        qq = __dp4a(a0, a0, qq);
        qq = __dp4a(a1, a1, qq);
        qq = __dp4a(b0, b0, qq);
        qq = __dp4a(b1, b1, qq);
        qx = __dp4a(a0, pa.x, qx);
        qx = __dp4a(a1, pa.y, qx);
        qx = __dp4a(b0, pb.x, qx);
        qx = __dp4a(b1, pb.y, qx);
    }
    if (dst != nullptr) {
        if constexpr (SMEM) {
            *reinterpret_cast<uint2 *>(dst + n * dpitch) = make_uint2(a0, a1);
            *reinterpret_cast<uint2 *>(dst + (8 + n) * dpitch) = make_uint2(b0, b1);
        } else {
            store_row_u8(dst + n * dpitch, dalign, a0, a1);
            if (has_b) store_row_u8(dst + (8 + n) * dpitch, dalign, b0, b1);
        }
    }
}

// Z = s W Y (s = +1 or -1) for the coefficients of zone KEEP (kept: rank < R,
// else dropped) of both blocks, as f32x2 pairs in units of 2^-149: one IMAD
// builds the bit pattern of 1.5 * 2^23 + s W y, one FMA rescales it exactly.
// Returns sum over the zone of W Y^2 for both blocks (per weight group in 32
// bits: at most 576 sum a^2 per block in all, so no group overflows).
template <int R, bool KEEP, int SIGN>
__device__ __forceinline__ unsigned long long zone_to_z(const int (&Ya)[8][8], const int (&Yb)[8][8], f2 (&Z)[8][8]) {
    unsigned g2[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    const f2 unit = f2_make(0x1p-149f, 0x1p-149f), bias = f2_make(-0x1.8p-126f, -0x1.8p-126f);
    static_for<0, 8>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<0, 8>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            if constexpr ((zz_rank(i, j) < R) == KEEP) {
                const int ya = Ya[i][j], yb = Yb[i][j];
                g2[weight_group(i, j)] += (unsigned)(ya * ya) + (unsigned)(yb * yb);
                constexpr int sw = SIGN * weight(i, j);
                const int za = ya * sw + 0x4B400000, zb = yb * sw + 0x4B400000;
                Z[i][j] = fma2(f2_make(__int_as_float(za), __int_as_float(zb)), unit, bias);
            }
        });
    });
    unsigned long long e = 0;
#pragma unroll
    for (int g = 0; g < 6; ++g) e += (unsigned long long)g2[g] * (unsigned)group_weight(g);
    return e;
}

// Column pass of the inverse over the zone's columns: U = C0^T Z.
template <int R, bool KEEP>
__device__ __forceinline__ void inverse_columns(const f2 (&Z)[8][8], f2 (&U)[8][8]) {
    static_for<0, 8>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        constexpr unsigned m = KEEP ? kept_col_mask(R, j) : drop_col_mask(R, j);
        if constexpr (m != 0u) {
            f2 in[8], out[8];
            static_for<0, 8>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if constexpr ((m >> i) & 1u) in[i] = Z[i][j];
                else in[i] = f2{0ull};
            });
            c0t_inverse<m>(in, out);
#pragma unroll
            for (int i = 0; i < 8; ++i) U[i][j] = out[i];
        }
    });
}

// Row n of the inverse's row pass: E = U[n] C0 over the zone's columns.
template <unsigned RM>
__device__ __forceinline__ void inverse_row(const f2 (&U)[8][8], int n, f2 (&E)[8]) {
    f2 in[8];
    static_for<0, 8>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if constexpr ((RM >> j) & 1u) in[j] = U[n][j];
        else in[j] = f2{0ull};
    });
    c0t_inverse<RM>(in, E);
}

// The two vertically adjacent blocks of a column pair at once, keeping
// exactly the first R zigzag coefficients (R is a compile-time constant, so
// the compiler drops every forward output, conversion and inverse term that
// the form in use never needs).  The forward transform and the compression
// run per block in int32, and from the compressed coefficients on every value
// is an f32x2 pair (block a, block b), so each inverse butterfly and each
// output scaling serves both blocks.  wb is all zeros when the pair has only
// its upper block (has_b false): a zero block contributes nothing to either
// error and is not stored.  Returns 576 * SSE of the two blocks (unrounded
// reconstruction); with E8 also adds the squared error of the 8-bit
// reconstruction to s8.  dst may be nullptr (errors only).  SMEM: dst is a
// shared-memory staging box (row pitch dpitch, 8-byte aligned rows) that a
// TMA store writes out, rather than the plane itself.  E8 is a compile-time
// choice so that kernels without the 8-bit error keep their registers.
template <int R, bool SMEM, bool E8>
__device__ __forceinline__ unsigned long long fused2_pair(const uint2 (&wa)[8], const uint2 (&wb)[8], uint8_t *dst,
                                                          int64_t dpitch, int dalign, bool has_b,
                                                          unsigned long long &s8) {
    const bool rec = E8 || dst != nullptr;
    unsigned qq = 0, qx = 0, sumsq = 0;
    if constexpr (R == 64) {
        // nothing is dropped: the reconstruction is the block itself, both errors are 0
        if (dst != nullptr) {
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                if constexpr (SMEM) {
                    *reinterpret_cast<uint2 *>(dst + n * dpitch) = wa[n];
                    *reinterpret_cast<uint2 *>(dst + (8 + n) * dpitch) = wb[n];
                } else {
                    store_row_u8(dst + n * dpitch, dalign, wa[n].x, wa[n].y);
                    if (has_b) store_row_u8(dst + (8 + n) * dpitch, dalign, wb[n].x, wb[n].y);
                }
            }
        }
        return 0ull;
    } else if constexpr (drop_form(R)) {
        int Ya[8][8], Yb[8][8];
        forward_pair<R>(wa, wb, Ya, Yb);
        // Z = -W Y on the dropped coefficients, so that the inverse yields -D
        f2 Z[8][8];
        const unsigned long long dropped = zone_to_z<R, false, -1>(Ya, Yb, Z);
        if (rec) {
            if constexpr (E8) sumsq = pair_sumsq(wa, wb);
            f2 U[8][8];
            inverse_columns<R, false>(Z, U);
            const f2 k576 = f2_make(576.0f, 576.0f);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                f2 E[8];
                inverse_row<drop_row_mask(R)>(U, n, E);
                // 576 Xhat = 576 A - D: a pixel as float bits is a * 2^-149 (exact,
                // subnormal), and the FMA forms 576 a - D exactly
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const unsigned wA = m < 4 ? wa[n].x : wa[n].y, wB = m < 4 ? wb[n].x : wb[n].y;
                    const f2 P = f2_make(__uint_as_float(byte_of(wA, m & 3)), __uint_as_float(byte_of(wB, m & 3)));
                    E[m] = fma2(P, k576, E[m]);
                }
                emit_row<SMEM, E8>(E, n, wa[n], wb[n], dst, dpitch, dalign, has_b, qq, qx);
            }
            if constexpr (E8) s8 += (unsigned long long)(sumsq + qq - 2u * qx);
        }
        return dropped;
    } else {
        sumsq = pair_sumsq(wa, wb);
        int Ya[8][8], Yb[8][8];
        forward_pair<R>(wa, wb, Ya, Yb);
        f2 Z[8][8];
        const unsigned long long kept = zone_to_z<R, true, 1>(Ya, Yb, Z);
        if (rec) {
            f2 U[8][8];
            inverse_columns<R, true>(Z, U);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                f2 E[8];
                inverse_row<kept_row_mask(R)>(U, n, E);
                emit_row<SMEM, E8>(E, n, wa[n], wb[n], dst, dpitch, dalign, has_b, qq, qx);
            }
            if constexpr (E8) s8 += (unsigned long long)(sumsq + qq - 2u * qx);
        }
        return 576ull * (unsigned long long)sumsq - kept;
    }
}

// ------------------------------------------------------------------ kernel

// Launch shape per r: 128 registers (four CTAs of 128 threads per SM) up to
// r = 34, 168 (three CTAs) above, and never more than kFused2MaxCtas CTAs per
// SM (see launch_staged).  Measured on a 600-frame 4K clip with the forward
// forms of packed_forward: four CTAs are 1.6 to 3.7% faster than three at
// r = 27..34, within 0.2% up to r = 26, and 1 to 5.5% slower at r = 35..40
// (two CTAs with 255 registers were 4-8% slower from r = 45 up).  Shared
// memory beyond four rings squeezes the L1 the copies go through.
template <int R, bool E8 = false>
struct Fused2Shape {
    static constexpr int threads = 128;
    // the 8-bit error's extra accumulators spill at 128 registers from r = 24
    static constexpr int min_blocks = R <= (E8 ? 23 : 34) ? 4 : 3;
};
constexpr int kStages = 2;   // cp.async ring depth per thread (double buffer)
constexpr int kVRows = kFusedVRows;  // vertically adjacent blocks per thread per strip
constexpr int kFused2MaxCtas = 4;    // CTAs per SM (measured best; leaves L1 for the copies)
constexpr int kFused2Smem = kStages * 8 * kVRows * 128 * 8;  // ring bytes per 128-thread CTA

__device__ __forceinline__ void cp_async8(uint32_t smem_addr, const void *gptr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Work description shared by the single-plane and batch launches.  Items are
// runs of 32 consecutive column pairs of a plane (see fused_items_of).
struct Fused2Args {
    const JobDesc *jobs;       // batch: device job table; single: unused
    const Chunk *chunks;       // batch: device chunk table; single: unused
    int32_t nchunks;
    int32_t chunk_items;       // single: items per virtual chunk
    unsigned long long *acc;   // batch: per-image 576*SSE; single: one slot
    unsigned long long *acc8;  // same slots for the squared error of the 8-bit reconstruction, or nullptr
    JobDesc single;            // single-plane job (by value)
};

template <bool SINGLE>
__device__ __forceinline__ Chunk get_chunk(const Fused2Args &a, int c) {
    if constexpr (SINGLE) {
        const int total = fused_items_of(a.single);
        const int it0 = c * a.chunk_items;
        const int n = total - it0 < a.chunk_items ? total - it0 : a.chunk_items;
        return Chunk{0, it0, n, a.single.r - 1};
    } else {
        return a.chunks[c];
    }
}
template <bool SINGLE>
__device__ __forceinline__ const JobDesc &get_job(const Fused2Args &a, int j) {
    if constexpr (SINGLE) return a.single;
    else return a.jobs[j];
}

// Walks the items of one warp: chunks c = warp, warp + nwarps, ...; each lane
// tracks its own column pair (row pair rp, block column bx), advanced by 32
// per item without divisions.
struct Cursor {
    int c, left, job, cls, rp, bx;
};
template <bool SINGLE>
__device__ __forceinline__ void cursor_load(const Fused2Args &a, Cursor &cu, int lane) {
    if (cu.c < a.nchunks) {
        const Chunk ch = get_chunk<SINGLE>(a, cu.c);
        const int nbw = get_job<SINGLE>(a, ch.job).nbw;
        const int L = ch.item0 * 32 + lane;
        cu.rp = L / nbw;
        cu.bx = L - cu.rp * nbw;
        cu.left = ch.nitems;
        cu.job = ch.job;
        cu.cls = ch.cls;
    }
}
template <bool SINGLE>
__device__ __forceinline__ void cursor_next(const Fused2Args &a, Cursor &cu, int nwarps, int lane) {
    if (--cu.left > 0) {
        const int nbw = get_job<SINGLE>(a, cu.job).nbw;
        cu.bx += 32;
        while (cu.bx >= nbw) {
            cu.bx -= nbw;
            ++cu.rp;
        }
    } else {
        cu.c += nwarps;
        cursor_load<SINGLE>(a, cu, lane);
    }
}

// Copy this lane's blocks (rows of block v at ring rows 8v .. 8v+7) into ring
// stage `st`.
template <int THREADS>
__device__ __forceinline__ void fetch_strip(const JobDesc &job, int rp, int bx, uint2 *ring, int st) {
    const int by = rp * kVRows;
    if (by < job.nbh) {
        const int64_t pitch = job.src_pitch;
        const uint8_t *src = job.src + (int64_t)by * 8 * pitch + (int64_t)bx * 8;
        uint2 *dst = ring + st * 8 * kVRows * THREADS + threadIdx.x;
        const int rows = (job.nbh - by) >= kVRows ? 8 * kVRows : 8 * (job.nbh - by);
        if (job.align >= 8) {
            const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(dst);
#pragma unroll
            for (int i = 0; i < 8 * kVRows; ++i) {
                if (i < rows) cp_async8(s0 + i * THREADS * 8, src);
                src += pitch;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8 * kVRows; ++i) {
                if (i < rows) {
                    uint2 v;
                    v.x = (uint32_t)src[0] | ((uint32_t)src[1] << 8) | ((uint32_t)src[2] << 16) |
                          ((uint32_t)src[3] << 24);
                    v.y = (uint32_t)src[4] | ((uint32_t)src[5] << 8) | ((uint32_t)src[6] << 16) |
                          ((uint32_t)src[7] << 24);
                    dst[i * THREADS] = v;
                }
                src += pitch;
            }
        }
    }
    cp_async_commit();
}

// Persistent fused kernel: each lane owns kVRows vertically adjacent blocks of
// every strip its warp visits; strips stream through a double-buffered
// per-thread cp.async ring.  CLO..CHI are the launch classes compiled in
// (class r - 1 keeps r coefficients; one class per launch).  E8: also the
// squared error of the 8-bit reconstruction (into a.acc8).
template <int CLO, int CHI, bool SINGLE, int THREADS, int MINB, bool E8>
__global__ void __launch_bounds__(THREADS, MINB) fused2_kernel(const Fused2Args a) {
    __shared__ uint2 ring[kStages * 8 * kVRows * THREADS];
    // The next launch of a batch (another r) may start as CTAs of this one
    // retire: the launches touch disjoint planes and only add into the error
    // slots.  Without a programmatic dependent launch this is a no-op.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);

    Cursor fc{gw, 0, 0, 0, 0, 0};
    cursor_load<SINGLE>(a, fc, lane);
    Cursor cc = fc;
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (fc.c < a.nchunks) {
            fetch_strip<THREADS>(get_job<SINGLE>(a, fc.job), fc.rp, fc.bx, ring, s);
            cursor_next<SINGLE>(a, fc, nwarps, lane);
        } else {
            cp_async_commit();
        }
    }
    unsigned long long s576 = 0, s8 = 0;
    int stage = 0;
    while (cc.c < a.nchunks) {
        cp_async_wait<kStages - 2>();
        const JobDesc &job = get_job<SINGLE>(a, cc.job);
        const int by = cc.rp * kVRows;
        const int nblk = by < job.nbh ? (job.nbh - by >= kVRows ? kVRows : job.nbh - by) : 0;
        const int refill = stage == 0 ? kStages - 1 : stage - 1;
        if (fc.c < a.nchunks) {
            fetch_strip<THREADS>(get_job<SINGLE>(a, fc.job), fc.rp, fc.bx, ring, refill);
            cursor_next<SINGLE>(a, fc, nwarps, lane);
        } else {
            cp_async_commit();
        }
        uint8_t *dst = job.dst ? job.dst + (int64_t)by * 8 * job.dst_pitch + (int64_t)cc.bx * 8 : nullptr;
        // both blocks of the column pair together (the lower one all zeros
        // when the plane ends after the upper one); lanes past the end of the
        // plane (nblk == 0) fetched nothing and do nothing
        if (nblk > 0) {
            static_assert(kVRows == 2, "fused2_pair handles two blocks");
            uint2 wa[8], wb[8];
            const bool has_b = nblk == 2;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                wa[i] = ring[((stage * kVRows + 0) * 8 + i) * THREADS + threadIdx.x];
                wb[i] = has_b ? ring[((stage * kVRows + 1) * 8 + i) * THREADS + threadIdx.x] : make_uint2(0u, 0u);
            }
            static_for<CLO, CHI + 1>([&](auto cc_) {
                constexpr int c = decltype(cc_)::value;
                if (cc.cls == c) s576 += fused2_pair<c + 1, false, E8>(wa, wb, dst, job.dst_pitch, job.dalign, has_b, s8);
            });
        }
        stage = stage + 1 == kStages ? 0 : stage + 1;
        const int img = job.image;
        const int cprev = cc.c;
        cursor_next<SINGLE>(a, cc, nwarps, lane);
        if (cc.c != cprev) {  // end of a chunk: one atomic per warp (and error)
            const unsigned long long t = warp_sum_u64(s576);
            if (lane == 0 && t) atomicAdd(SINGLE ? a.acc : a.acc + img, t);
            s576 = 0;
            if constexpr (E8) {
                const unsigned long long t8 = warp_sum_u64(s8);
                if (lane == 0 && t8) atomicAdd(SINGLE ? a.acc8 : a.acc8 + img, t8);
                s8 = 0;
            }
        }
    }
    cp_async_wait<0>();
    // Complete only after the launch this one overlapped has completed, so
    // that whatever follows the last launch of a batch in stream order sees
    // every launch's errors.
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------ TMA staging
//
// Batch plans whose planes all start on 16-byte boundaries with 16-byte
// pitches stage their pixels with the tensor memory accelerator instead of
// per-thread copies.  A work item is then one row pair x a segment of 32
// column pairs starting at a multiple of 32 columns, i.e. one 256 x 16-byte
// box of the plane, which one lane requests with cp.async.bulk.tensor (the
// box's columns and rows outside the plane arrive as zeros); each warp has a
// two-stage ring of boxes and one mbarrier per stage.
constexpr int kTmaBoxW = 256, kTmaBoxH = 16, kTmaBoxBytes = kTmaBoxW * kTmaBoxH;

struct TmaArgs {
    const JobDesc *jobs;
    const Chunk *chunks;        // items: row pair * segments + segment
    const unsigned char *maps;  // per job: the source plane's tensor map, then the destination's
    int32_t nchunks;
    unsigned long long *acc;    // per-image 576 * SSE
    unsigned long long *acc8;   // per-image squared error of the 8-bit reconstruction, or nullptr
};

__device__ unsigned int g_tma_timeouts = 0;

__device__ __forceinline__ bool tma_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One lane: write a staged box of the reconstruction to the plane (rows and
// columns outside the plane are dropped) and close the bulk group.
__device__ __forceinline__ void tma_store(const unsigned char *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
                 "r"(y), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// One lane: wait until the shared memory of every committed store was read.
__device__ __forceinline__ void tma_store_drain_reads() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// One lane: expect the box's bytes on the stage's mbarrier and request it.
__device__ __forceinline__ void tma_request(const unsigned char *map, uint32_t dst, uint32_t mbar, int x, int y) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "n"(kTmaBoxBytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// TSTORE: the reconstruction goes out through the box with TMA stores, else
// with per-thread stores straight from registers.  E8 as for fused2_kernel.
template <int CLS, int THREADS, int MINB, bool TSTORE, bool E8>
__global__ void __launch_bounds__(THREADS, MINB) fused2_tma_kernel(const TmaArgs a) {
    constexpr int WARPS = THREADS / 32;
    __shared__ __align__(128) unsigned char boxes[WARPS * kStages * kTmaBoxBytes];
    __shared__ __align__(8) unsigned long long bars[WARPS * kStages];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarps = (int)(gridDim.x * WARPS);
    const int gw = (int)(blockIdx.x * WARPS + wid);
    const uint32_t ring = (uint32_t)__cvta_generic_to_shared(boxes + wid * kStages * kTmaBoxBytes);
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[wid * kStages]);
    if (lane == 0) {
#pragma unroll
        for (int st = 0; st < kStages; ++st) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * st));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // the warp's items, in order: chunks gw, gw + nwarps, ..., each item0 .. item0 + nitems - 1
    // (c, left, rp, seg): the next item to request; an item's row pair and
    // segment are divided out once per chunk and then stepped
    int c = gw, left = 0, rp = 0, seg = 0, segs = 1;
    Chunk ch{};
    auto load_chunk = [&]() {
        if (c < a.nchunks) {
            ch = a.chunks[c];
            segs = a.jobs[ch.job].segs;
            rp = ch.item0 / segs;
            seg = ch.item0 - rp * segs;
            left = ch.nitems;
        }
    };
    auto advance = [&]() {
        if (--left > 0) {
            if (++seg == segs) {
                seg = 0;
                ++rp;
            }
        } else {
            c += nwarps;
            load_chunk();
        }
    };
    auto request = [&](int st) {  // the next item into stage st
        if (lane == 0)
            tma_request(a.maps + (int64_t)ch.job * 2 * kTensorMapBytes, ring + st * kTmaBoxBytes, bar0 + 8 * st,
                        seg * kTmaBoxW, rp * kTmaBoxH);
    };

    load_chunk();
    if (c >= a.nchunks) return;
    request(0);
    int cur_c = c, crp = rp, cseg = seg;  // the item in flight in `stage`
    Chunk cch = ch;
    advance();
    uint32_t phase = 0u;           // bit st: parity of stage st's next completion
    unsigned long long s576 = 0, s8 = 0;
    int stage = 0;
    while (true) {
        const bool more = c < a.nchunks;
        if (more) {  // the other stage was read (and stored from) in the previous iteration
            __syncwarp();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (lane == 0) tma_store_drain_reads();
            request(stage ^ 1);
        }
        const bool got = tma_wait(bar0 + 8 * stage, (phase >> stage) & 1u);
        phase ^= 1u << stage;
        if (!__all_sync(0xffffffffu, got)) {
            if (lane == 0) atomicAdd(&g_tma_timeouts, 1u);
            if (more) tma_wait(bar0 + 8 * (stage ^ 1), (phase >> (stage ^ 1)) & 1u);
            break;
        }
        const JobDesc &job = a.jobs[cch.job];
        const int bx = cseg * 32 + lane, by = 2 * crp;
        unsigned char *box = boxes + (wid * kStages + stage) * kTmaBoxBytes;
        const bool store = TSTORE && job.dst != nullptr;
        if (bx < job.nbw) {
            uint2 wa[8], wb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                wa[i] = *reinterpret_cast<const uint2 *>(box + i * kTmaBoxW + lane * 8);
                wb[i] = *reinterpret_cast<const uint2 *>(box + (8 + i) * kTmaBoxW + lane * 8);
            }
            const bool has_b = by + 1 < job.nbh;
            if constexpr (TSTORE) {
                // the reconstruction replaces the pixels in the box (each lane its own columns)
                s576 += fused2_pair<CLS + 1, true, E8>(wa, wb, store ? box + lane * 8 : nullptr, kTmaBoxW, 8, has_b,
                                                       s8);
            } else {
                uint8_t *dst = job.dst ? job.dst + (int64_t)by * 8 * job.dst_pitch + (int64_t)bx * 8 : nullptr;
                s576 += fused2_pair<CLS + 1, false, E8>(wa, wb, dst, job.dst_pitch, job.dalign, has_b, s8);
            }
        }
        if (store) {  // one TMA store of the box; columns and rows outside the plane are dropped
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                tma_store(a.maps + (int64_t)cch.job * 2 * kTensorMapBytes + kTensorMapBytes,
                          (uint32_t)__cvta_generic_to_shared(box), cseg * kTmaBoxW, crp * kTmaBoxH);
        }
        if (!more || c != cur_c) {  // the item closed its chunk: one atomic per warp and chunk (and error)
            const unsigned long long t = warp_sum_u64(s576);
            if (lane == 0 && t) atomicAdd(a.acc + job.image, t);
            s576 = 0;
            if constexpr (E8) {
                const unsigned long long t8 = warp_sum_u64(s8);
                if (lane == 0 && t8) atomicAdd(a.acc8 + job.image, t8);
                s8 = 0;
            }
        }
        if (!more) break;
        cur_c = c;
        crp = rp;
        cseg = seg;
        cch = ch;
        advance();
        stage ^= 1;
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores done before exit
    __syncwarp();
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// TMA stores of the reconstruction pay where instruction issue binds (they
// replace sixteen per-thread stores and their address arithmetic per item):
// measured +3.5% at r = 21 and +4.6% at r = 32, but 1% slower at r = 16.
constexpr bool tma_store_pays(int R) { return R > 16; }

// TMA-staged batch launch for exactly r = R (instantiated with the others).
template <int R>
cudaError_t launch_fused2_tma_r(const TmaArgs &a, int ctas_per_sm, bool overlap, cudaStream_t s) {
    constexpr int T = Fused2Shape<R>::threads, MB = Fused2Shape<R>::min_blocks, MB8 = Fused2Shape<R, true>::min_blocks;
    constexpr bool TS = tma_store_pays(R);
    constexpr int smem = (T / 32) * kStages * kTmaBoxBytes;
    if (a.acc8 != nullptr)
        return launch_staged(fused2_tma_kernel<R - 1, T, MB8, TS, true>, a.nchunks, ctas_per_sm, T / 32,
                             kFused2MaxCtas, smem, overlap, s, a);
    return launch_staged(fused2_tma_kernel<R - 1, T, MB, TS, false>, a.nchunks, ctas_per_sm, T / 32, kFused2MaxCtas,
                         smem, overlap, s, a);
}

// Launch for exactly r = R retained coefficients: single-plane (a.single) or
// batch (a.jobs / a.chunks).  Instantiated per R in rdct_fused2_r*.cu.
// overlap: a programmatic dependent launch on the previous kernel of the
// stream (batch launches after the first of a batch).
template <int R>
cudaError_t launch_fused2_r(const Fused2Args &a, bool single, int ctas_per_sm, bool overlap, cudaStream_t s) {
    constexpr int T = Fused2Shape<R>::threads, MB = Fused2Shape<R>::min_blocks, MB8 = Fused2Shape<R, true>::min_blocks;
    const bool e8 = a.acc8 != nullptr;
    if (single)
        return e8 ? launch_staged(fused2_kernel<R - 1, R - 1, true, T, MB8, true>, a.nchunks, ctas_per_sm, T / 32,
                                  kFused2MaxCtas, kFused2Smem, false, s, a)
                  : launch_staged(fused2_kernel<R - 1, R - 1, true, T, MB, false>, a.nchunks, ctas_per_sm, T / 32,
                                  kFused2MaxCtas, kFused2Smem, false, s, a);
    return e8 ? launch_staged(fused2_kernel<R - 1, R - 1, false, T, MB8, true>, a.nchunks, ctas_per_sm, T / 32,
                              kFused2MaxCtas, kFused2Smem, overlap, s, a)
              : launch_staged(fused2_kernel<R - 1, R - 1, false, T, MB, false>, a.nchunks, ctas_per_sm, T / 32,
                              kFused2MaxCtas, kFused2Smem, overlap, s, a);
}

}  // namespace rdct
