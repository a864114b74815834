// rdct_tc.cuh -- tensor-core pieces of the kernels that transform 128 blocks
// at a time as one product D = A B^T (the DCT pass of the r sweep).
//
// A (128 x 64, FP16): one block per row, its 64 pixels in row-major order
// (k = 8 y + x); each thread writes its own block into its own lane of tensor
// memory with tcgen05.st (32 columns of FP16 pairs).  B (64 x 64, FP16) sits
// in shared memory in the K-major layout without swizzle: 8 x 8 core matrices
// of 16-byte rows, K-adjacent core matrices 128 bytes apart, 8-row groups
// 1 KB apart.  For a separable 2-D transform Y = F A F^T, row n = 8 i + j of
// B holds F[i][y] F[j][x], so D's row b holds the coefficients of block b.  A
// B that is not exact in FP16 enters as the sum of two FP16 matrices (the
// high part and the rest), accumulated into the same FP32 result.
//
// Tensor memory of a group of 128 threads: A in its columns 0..31, D in
// 64..127; four groups per CTA use all 512 columns of an SM.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

namespace rdct {
namespace tc {

constexpr int kGroup = 128;                      // threads (and blocks) of a group: the MMA's M
constexpr int kGroups = 4;                       // groups per CTA, one CTA per SM
constexpr int kThreads = kGroup * kGroups;
constexpr uint32_t kGroupCols = 128;             // tensor-memory columns per group
constexpr uint32_t kCols = kGroupCols * kGroups;  // all 512
constexpr uint32_t kDCol = 64;                   // D's first column within the group's columns
constexpr uint32_t kLbo = 128, kSbo = 8 * 128;   // K-adjacent core matrices, 8-row groups
constexpr uint32_t kBBytes = 64 * 64 * 2;        // one 64 x 64 FP16 matrix
constexpr int kWaitPolls = 1 << 22;              // bound of every mbarrier wait

// Shared-memory matrix descriptor (no swizzle, K-major).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kSbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Byte offset of element (row n, column k) of a 64 x 64 FP16 matrix in that layout.
__device__ __forceinline__ uint32_t core_off(int n, int k) {
    return (uint32_t)((n >> 3) * kSbo + (k >> 3) * kLbo + (n & 7) * 16 + (k & 7) * 2);
}
// Instruction descriptor: D FP32, A and B FP16, both K-major, N = 64, M = 128.
constexpr uint32_t kIdescM128N64 = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// B = F (x) F for the 8 x 8 matrix f (row-major FP32), as NB FP16 parts
// (NB = 1: f (x) f must be exact in FP16; NB = 2: high part and rest) at
// bsm, bsm + kBBytes.  Called by every thread of the CTA.
template <int NB>
__device__ __forceinline__ void build_kron_b(unsigned char *bsm, const float *f, int tid, int nthreads) {
    for (int e = tid; e < 64 * 64; e += nthreads) {
        const int n = e >> 6, k = e & 63, i = n >> 3, j = n & 7, y = k >> 3, x = k & 7;
        const float c = f[i * 8 + y] * f[j * 8 + x];
        const __half hi = __float2half_rn(c);
        *reinterpret_cast<__half *>(bsm + core_off(n, k)) = hi;
        if constexpr (NB == 2)
            *reinterpret_cast<__half *>(bsm + kBBytes + core_off(n, k)) = __float2half_rn(c - __half2float(hi));
    }
}

// Barrier of the 128 threads of group g (named barrier 1 + g), and the same
// barrier reducing a flag with OR.
__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(kGroup) : "memory");
}
__device__ __forceinline__ bool group_sync_or(int g, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + g), "n"(kGroup)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tmem_alloc_all(uint32_t *slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc_all(uint32_t base) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(kCols));
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 columns of this warp's 32 lanes (lane = thread): store and load.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&a)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]),
        "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// The 16x256b fragment, four 8-column repetitions: lane l receives columns
// 8 k + 2 (l mod 4) + {0, 1} (k = 0..3) of rows l/4 and l/4 + 8 of the 16
// lanes at taddr, as r[4 k + 2 row + e].
__device__ __forceinline__ void tmem_ld_frag(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Pixels (x, x + 1) of a row word as an FP16 pair a - BIAS: the byte goes
// under the FP16 exponent of 1024 (high byte 0x64), then 1024 + BIAS is
// subtracted -- exact for BIAS = 0 or 128.
template <int BIAS>
__device__ __forceinline__ uint32_t px_pair(uint32_t word, int x) {
    static_assert(BIAS == 0 || BIAS == 128, "bias");
    const unsigned b = (unsigned)(x & 3);
    const uint32_t t = __byte_perm(word, 0x64646464u, b | (4u << 4) | ((b + 1u) << 8) | (4u << 12));
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(t), "r"(BIAS == 0 ? 0x64006400u : 0x64806480u));
    return d;
}
// A block's 64 pixels (w[2 y], w[2 y + 1] = row y) into this thread's lane of
// A at column a_col: the FP16 pair (x, x + 1) of row y in column 4 y + x / 2.
template <int BIAS>
__device__ __forceinline__ void store_block_a(uint32_t a_col, const uint32_t (&w)[16]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t a[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int k = 2 * (16 * h + c), y = k >> 3, x = k & 7;
            a[c] = px_pair<BIAS>(w[2 * y + (x >> 2)], x);
        }
        tmem_st16(a_col + 16u * h, a);
    }
}

// D (at column d) = A (at column a) B^T over K = 64, B as NB FP16 parts at
// shared address sb; then one arrive on the mbarrier when they are done.
// Issued by one thread.
template <int NB>
__device__ __forceinline__ void mma_tile(uint32_t d, uint32_t a, uint32_t sb, uint32_t mbar) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            const uint64_t bd = smem_desc(sb + (uint32_t)m * kBBytes + (uint32_t)kk * 2u * kLbo);
            const uint32_t acc = (kk > 0 || m > 0) ? 1u : 0u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
                         "r"(a + 8u * (uint32_t)kk), "l"(bd), "r"(kIdescM128N64), "r"(acc));
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// Bounded wait for the mbarrier phase of the given parity; true when it completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kWaitPolls && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    return done != 0;
}
// The same with test_wait (no suspend), for the exit path after a timeout.
__device__ __forceinline__ bool mbar_test_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kWaitPolls && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    return done != 0;
}
__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

}  // namespace tc
}  // namespace rdct
