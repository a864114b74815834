// rdct_sweep_tc.cu -- the DCT pass of the r sweep (Sec. 3: SSE for every r,
// for the exact DCT the paper compares against) with the block transforms on
// the tensor cores.
//
// The sweep needs, per plane and coefficient position q, the energy
// E_q = sum over blocks of Y_q^2.  For a tile of 128 blocks the coefficients
// of every block are one product  D = A B^T:  A (128 x 64) holds the blocks'
// pixels, one block per row (the MMA's M), B (64 x 64) the transform of the
// 64 pixels into the 64 coefficients (row q = 8 i + j: the entries
// C[i][y] C[j][x]), so D[b][q] = Y_q of block b.  Each thread owns one block:
// it writes the block's pixels as FP16 straight into its own lane of tensor
// memory (tcgen05.st; the A operand of tcgen05.mma may live there), and one
// thread issues the MMAs with B from shared memory.  The coefficients come
// back in the 16x256b fragment of tcgen05.ld: lane l of a warp holds
// columns 8k + 2(l mod 4) + {0, 1} of rows l/4 and l/4 + 8 of each 16-row
// half of the warp's 32 rows, so each thread keeps 16 energy bins (for
// four blocks) instead of 64.  No pixel passes through shared memory.
//
// The time goes to the chain of each tile (stores into tensor memory, group
// barrier, MMAs, their commit, loads back): on the 1024 x 512^2 batch, with
// one wait per load back (92 us per call), copies of the kernel without its
// global loads took 78 us, without its MMAs (and the wait for them) 65,
// without both 47.  Overlapping one tile's MMAs with the previous tile's
// read-back needs two D buffers per group, and so fewer groups (three,
// 98 us) or A in shared memory (94 us); deeper load prefetch, in registers
// or through a cp.async ring, was slower as well (100-115 us), and so were a
// single thread waiting for the MMAs instead of all (88 us) and six groups
// per SM with A in shared memory (89 us).
//
// The pixels enter centred, a - 128 (exact in FP16; every AC row of C (x) C
// sums to zero, so the AC coefficients do not change, and the DC coefficient
// is never needed: every r keeps it).  C (x) C enters as the sum of two FP16
// matrices (hi and lo parts) accumulated into the same FP32 result, which
// keeps the coefficients at FP32 accuracy; FP32 bins per thread, FP64 plane
// bins.  (The RDCT pass stays on the per-block kernel: in this form each of
// its coefficients needs an exact conversion and an integer multiply-add
// where the DCT needs one FFMA, and it measured 123 us against 102 us per
// call on 1024 x 512^2.)
//
// Work: a flat list of tiles over the planes (JobDesc::pad = the plane's first
// tile, non-decreasing).  One CTA per SM of four independent groups of 128
// threads; each group owns a quarter of the SM's tensor memory (A in its
// columns 0..31, D in 64..127), its own mbarrier and named barrier, and a
// contiguous range of tiles, and loads its next tile before the current
// tile's MMAs.  (With one 128-thread CTA per group the block scheduler kept
// fewer groups per SM busy than their resources allow.)
#include <cuda_runtime.h>

#include <cstdint>

#include "rdct_blocks.cuh"
#include "rdct_device.cuh"
#include "rdct_internal.h"
#include "rdct_tc.cuh"

namespace rdct {
namespace {

using tc::kGroup;
constexpr int kTcFlushTiles = 32;  // tiles (4 blocks each) summed in FP32 per bin before the FP64 plane bins

__device__ unsigned int g_sweep_tc_timeouts = 0;

struct TcPlane {
    int idx, base, end;  // plane index, its first tile, one past its last
    const uint8_t *src;
    int64_t pitch;
    int nbw, nblocks, align;
};
__device__ __forceinline__ void tc_plane_load(const JobDesc *jobs, int n, int total, int idx, TcPlane &p) {
    const JobDesc &j = jobs[idx];
    p.idx = idx;
    p.base = j.pad;
    p.end = idx + 1 < n ? jobs[idx + 1].pad : total;
    p.src = j.src;
    p.pitch = j.src_pitch;
    p.nbw = j.nbw;
    p.nblocks = j.nbw * j.nbh;
    p.align = j.align;
}
__device__ __forceinline__ void tc_plane_seek(const JobDesc *jobs, int n, int total, int u, TcPlane &p) {
    if (u < p.end) return;
    int idx = p.idx;
    while (idx + 1 < n && jobs[idx + 1].pad <= u) ++idx;
    tc_plane_load(jobs, n, total, idx, p);
}

// The loads' cursor: this thread's block (row by, column bx) in the tile being
// loaded, stepped by one tile (128 blocks) at a time; a division only when the
// plane changes.
struct TcCursor {
    TcPlane p;
    int by, bx, sq, sr;  // block position; 128 / nbw, 128 mod nbw
};
__device__ __forceinline__ void tc_cursor_init(TcCursor &c, int u, int gt) {
    const int b = (u - c.p.base) * kGroup + gt;
    c.by = b / c.p.nbw;
    c.bx = b - c.by * c.p.nbw;
    c.sq = kGroup / c.p.nbw;
    c.sr = kGroup - c.sq * c.p.nbw;
}
__device__ __forceinline__ void tc_cursor_next(const JobDesc *jobs, int n, int total, int u, int gt, TcCursor &c) {
    if (u >= c.p.end) {
        tc_plane_seek(jobs, n, total, u, c.p);
        tc_cursor_init(c, u, gt);
        return;
    }
    c.bx += c.sr;
    c.by += c.sq;
    if (c.bx >= c.p.nbw) {
        c.bx -= c.p.nbw;
        c.by += 1;
    }
}
// This thread's block at the cursor (16 words, rows in order), or `fill` words past the plane's end.
__device__ __forceinline__ void tc_load(const TcCursor &c, uint32_t fill, uint32_t (&w)[16]) {
    if (c.by * c.p.nbw + c.bx < c.p.nblocks) {
        load_block(c.p.src + (int64_t)c.by * 8 * c.p.pitch + (int64_t)c.bx * 8, c.p.pitch, c.p.align, w);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] = fill;
    }
}

// The warp's bins into the plane's zigzag bins.  Bin 2k + e of lane l holds
// coefficient (k, 2(l mod 4) + e); its total is the sum over the eight lanes
// with the same l mod 4, and lane l adds the totals of row k = l/4: two
// atomics per lane, the 64 positions of the block once each (DC skipped).
__device__ __forceinline__ void tc_flush(double *plane_bins, float (&fb)[16], int lane) {
    const int c = lane & 3, kl = lane >> 2;
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float v = fb[2 * k + e];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (k == kl) {
                if (e == 0) s0 = v;
                else s1 = v;
            }
            fb[2 * k + e] = 0.0f;
        }
    }
    if (s0 != 0.0f && (kl | c) != 0) atomicAdd(plane_bins + zz_rank(kl, 2 * c), (double)s0);
    if (s1 != 0.0f) atomicAdd(plane_bins + zz_rank(kl, 2 * c + 1), (double)s1);
}

__global__ void __launch_bounds__(tc::kThreads, 1)
    sweep_dct_tc_kernel(const JobDesc *__restrict__ jobs, int32_t nplanes, int32_t total, double *out,
                        const DctConsts C) {
    constexpr int NB = 2;  // B matrices: the hi and lo parts of C (x) C
    __shared__ __align__(1024) unsigned char bsm[NB * tc::kBBytes];
    __shared__ uint64_t bars[tc::kGroups];
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp >> 2, gt = tid & (kGroup - 1);
    // this group's tiles [t0, t1)
    const int64_t ngroups = (int64_t)gridDim.x * tc::kGroups, gi = (int64_t)blockIdx.x * tc::kGroups + g;
    const int t0 = (int)(gi * total / ngroups);
    const int t1 = (int)((gi + 1) * total / ngroups);
    tc::build_kron_b<NB>(bsm, C.c, tid, tc::kThreads);  // row n = 8 i + j (coefficient), column k = 8 y + x (pixel)
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(bsm);
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&bars[g]);
    if (warp == 0) tc::tmem_alloc_all(&slot);
    if (gt == 0) tc::mbar_init(mbar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B, written by these threads, is read by the MMAs
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // launched as a programmatic dependent of the table builder (which also
    // clears the bins): the set-up above overlaps the builder's tail
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t tb = *reinterpret_cast<volatile uint32_t *>(&slot) + tc::kGroupCols * (uint32_t)g;  // group's columns
    const uint32_t my_lane = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t fill = 0x80808080u;  // a missing block reads as 128 everywhere: zero once centred

    bool failed = false;
    int last_issued = -1;  // tiles of this group whose MMAs were issued: t0 .. last_issued
    if (t0 < t1) {
        float fb[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) fb[p] = 0.0f;
        TcPlane cur{};
        {
            int lo = 0, hi = nplanes - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].pad <= t0) lo = mid;
                else hi = mid - 1;
            }
            tc_plane_load(jobs, nplanes, total, lo, cur);
        }
        TcCursor ld{cur, 0, 0, 0, 0};
        tc_cursor_init(ld, t0, gt);
        uint32_t w[16];
        tc_load(ld, fill, w);
        int since_flush = 0;
        for (int u = t0; u < t1; ++u) {
            tc_plane_seek(jobs, nplanes, total, u, cur);
            tc::store_block_a<128>(my_lane, w);  // this thread's block, centred, into its lane of A
            tc::tmem_wait_st();
            // the next tile's block: its loads run while this tile is transformed
            if (u + 1 < t1) {
                tc_cursor_next(jobs, nplanes, total, u + 1, gt, ld);
                tc_load(ld, fill, w);
            }
            tc::fence_before_sync();
            tc::group_sync(g);
            tc::fence_after_sync();
            if (gt == 0) tc::mma_tile<NB>(tb + tc::kDCol, tb, sb, mbar);
            last_issued = u;
            // wait (bounded) for the MMAs; a group whose wait runs out stops after this tile
            const bool done = tc::mbar_wait(mbar, (uint32_t)(u - t0) & 1u);
            if (tc::group_sync_or(g, !done)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            // the coefficients of four blocks (rows l/4, l/4 + 8 of each 16-row half), 16 positions each,
            // in four loads and one wait: squares into the bins (the DC squares land in bin 0 of lanes
            // l mod 4 = 0 and are not flushed)
            {
                uint32_t r[4][16];  // r[2 half + kh][4 kk + 2 row + e]: column 8 (4 kh + kk) + 2 (l mod 4) + e
#pragma unroll
                for (int half = 0; half < 2; ++half)
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh)
                        tc::tmem_ld_frag(my_lane + ((uint32_t)(16 * half) << 16) + tc::kDCol + 32u * (uint32_t)kh,
                                         r[2 * half + kh]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int half = 0; half < 2; ++half)
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                            for (int row = 0; row < 2; ++row)
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const float y = __uint_as_float(r[2 * half + kh][4 * kk + 2 * row + e]);
                                    float &b = fb[2 * (4 * kh + kk) + e];
                                    b = __fmaf_rn(y, y, b);
                                }
            }
            tc::fence_before_sync();
            // flush at the end of the plane (for this group) or after kTcFlushTiles tiles
            ++since_flush;
            if (u + 1 == t1 || u + 1 >= cur.end || since_flush == kTcFlushTiles) {
                tc_flush(out + (int64_t)cur.idx * 64, fb, lane);
                since_flush = 0;
            }
            // (the next tile's group barrier, before its MMAs, orders every thread's reads of D before they are
            // overwritten)
        }
    }
    if (failed) {
        if (gt == 0) atomicAdd(&g_sweep_tc_timeouts, 1u);
        // the MMAs of the tile that timed out may still run: wait (bounded) before releasing the memory
        tc::mbar_test_wait(mbar, (uint32_t)(last_issued - t0) & 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc_all(*reinterpret_cast<volatile uint32_t *>(&slot));
}

}  // namespace

// One CTA per SM: each allocates all 512 tensor-memory columns (four groups
// of 128), and its launch bounds (128 registers for 512 threads) allow no
// second CTA on the SM.
cudaError_t launch_sweep_dct_tc(const JobDesc *jobs, int32_t nplanes, int32_t total_tiles, double *out,
                                cudaStream_t s) {
    if (total_tiles <= 0) return cudaSuccess;
    const int64_t g = sm_count();
    const int64_t need = (total_tiles + tc::kGroups - 1) / tc::kGroups;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g < need ? g : need));
    cfg.blockDim = dim3(tc::kThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sweep_dct_tc_kernel, jobs, nplanes, total_tiles, out, make_dct_consts());
}

unsigned int take_sweep_tc_timeouts() {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_sweep_tc_timeouts, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_sweep_tc_timeouts, &zero, sizeof(zero));
    }
    return v;
}

}  // namespace rdct
