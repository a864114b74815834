// rdct_sweep2.cuh -- the RDCT pass of the r sweep of Sec. 3, one pass per plane.
//
// The transforms are orthogonal (Sec. 2), so the squared error of the
// reconstruction that keeps the first r zigzag coefficients is the energy of
// the dropped orthonormal coefficients (Parseval).  One pass per plane
// therefore gives the error for every r: each thread transforms its blocks,
// adds every coefficient's energy into 64 per-position bins held in
// registers, and once per chunk the warp reduces the bins and adds them to the
// plane's 64 zigzag-ordered bins; suffix sums then give SSE(r), r = 1..64.
//
// Y = C0 A C0^T exactly (dp4a row pass on packed pixels, int32 column
// butterfly); the orthonormal energy of Y_ij is W_ij Y_ij^2 / 576, so the bins
// hold integer Y^2 sums (exact) and the weights are applied at the flush.
// Staging, strip cursors and chunking are those of the fused kernel.  (The
// exact DCT's pass runs on the tensor cores, in rdct_sweep_tc.cu.)
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
__device__ __forceinline__ void sweep_flush(double *plane_bins, unsigned (&ub)[64], int lane) {
    unsigned long long u0 = 0ull, u1 = 0ull;
#pragma unroll
    for (int p = 1; p < 64; ++p) {
        const unsigned long long s = warp_sum_u32_wide(ub[p]) * (unsigned)weight(p >> 3, p & 7);
        if (lane == (p & 31)) {
            if (p < 32) u0 = s;
            else u1 = s;
        }
        ub[p] = 0u;
    }
    const int k0 = kSweepZz.r[lane], k1 = kSweepZz.r[32 + lane];
    unsigned long long *b = reinterpret_cast<unsigned long long *>(plane_bins);
    if (u0) atomicAdd(b + k0, u0);
    if (u1) atomicAdd(b + k1, u1);
}

// Persistent sweep kernel over a chunk table (job = plane; out = [planes][64]
// zigzag-ordered bins of uint64 576-scaled energies; the DC bin stays 0).  Each warp takes a contiguous run of chunks, so that
// consecutive chunks mostly belong to one plane and the bins are flushed only
// when the plane changes or after kSweepFlushChunks chunks.
__global__ void __launch_bounds__(128, 4) sweep2_kernel(const Fused2Args args, double *out) {
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
#pragma unroll
    for (int p = 0; p < 64; ++p) ub[p] = 0u;
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
        // both blocks unrolled so that their work interleaves
#pragma unroll
        for (int v = 0; v < kVRows; ++v) {
            if (v < nblk) {
                uint2 w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w[i] = ring[((stage * kVRows + v) * 8 + i) * THREADS + threadIdx.x];
                sweep_rdct_block(w, ub);
            }
        }
        stage = stage + 1 == kStages ? 0 : stage + 1;
        const int plane = cc.job;
        const int cprev = cc.c;
        cursor_next<false>(a, cc, 1, lane);
        if (cc.c != cprev) {
            if (++since_flush == kSweepFlushChunks || cc.c >= a.nchunks || cc.job != plane) {
                sweep_flush(out + (int64_t)plane * 64, ub, lane);
                since_flush = 0;
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace rdct
