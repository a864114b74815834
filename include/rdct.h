/*
 * rdct.h -- C-ABI of librdct, a GB300 (sm_103a) library for the block image
 * codec built on the round-off DCT approximation of Cintra & Bayer, "A DCT
 * Approximation for Image Compression".
 *
 * The method (Sec. 2-3 of the paper):
 *   C0 = [2C]      the 8-point DCT matrix scaled by 2 and rounded (entries 0, +-1)
 *   S  = sqrt((C0 C0^T)^-1) = diag(1/(2 sqrt2), 1/sqrt6, 1/2, 1/sqrt6, ...)
 *   C_orth = S C0  (orthogonal)
 *   per 8x8 block A:  Y = C0 A C0^T  (additions only)
 *                     Yhat = first r zigzag coefficients of S Y S (S folded
 *                            into the compression step), the rest zeroed
 *                     Xhat = C_orth^T Yhat C_orth = C0^T S Yhat S C0
 *   quality: SSE / MSE / PSNR of Xhat against A.
 *
 * Conventions shared by every call:
 *   - Every call returns an rdct_status; no C++ exception crosses this ABI.
 *     rdct_status_string() names a status; rdct_last_error() copies the
 *     calling thread's last detailed message.
 *   - Data pointers are DEVICE pointers owned by the caller unless a
 *     parameter says "host".  The library never frees caller memory.
 *   - Calls that take an rdct_stream (a cudaStream_t; NULL = legacy default
 *     stream) are asynchronous on that stream.  Arguments are validated
 *     synchronously before anything is launched (RDCT_ERR_ARG /
 *     RDCT_ERR_SHAPE with nothing enqueued).  Errors raised by a kernel
 *     surface as RDCT_ERR_CUDA from this or a later call, or from rdct_sync.
 *   - Planes are 8-bit, row-major, with a pitch in bytes >= width.  Width
 *     and height must be positive multiples of 8 (the paper's images are
 *     512 x 512; other sizes are rejected, RDCT_ERR_SHAPE).  Multi-channel
 *     images are passed as separate planes.
 *   - Coefficient blocks are block-major: block (by, bx) of a plane with
 *     nbw = w/8 blocks per row is block index by * nbw + bx; within a block
 *     the 64 values are row-major (row = vertical frequency).
 *   - Zigzag order is the JPEG scan (first step horizontal): (0,0), (0,1),
 *     (1,0), (2,0), (1,1), (0,2), ...  This is the reading taken of the
 *     paper's "standard zigzag sequence" (Sec. 3).
 *   - Rounding to 8 bits: clamp(round(x), 0, 255), nearest integer; the
 *     integer path of rdct_fused rounds exact halves upward, the others
 *     round them to even.  Results may differ by 1 at exact halves.
 */
#ifndef RDCT_H
#define RDCT_H

#include <stddef.h>
#include <stdint.h>

#if defined(RDCT_BUILD) && defined(__GNUC__)
#define RDCT_API __attribute__((visibility("default")))
#else
#define RDCT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RDCT_OK = 0,
    RDCT_ERR_ARG = 1,        /* bad pointer, count or parameter */
    RDCT_ERR_SHAPE = 2,      /* width/height not a positive multiple of 8, pitch < width */
    RDCT_ERR_OOM = 3,        /* a device or pinned-host allocation failed */
    RDCT_ERR_TOO_LARGE = 4,  /* request larger than a configured budget or limit */
    RDCT_ERR_CUDA = 5,       /* a CUDA runtime call or kernel failed */
    RDCT_ERR_TIMEOUT = 6,    /* a wait ran out before the work completed */
    RDCT_ERR_BUSY = 7,       /* queue full; retry later */
    RDCT_ERR_NOT_FOUND = 8,  /* unknown ticket or handle, unreadable file */
    RDCT_ERR_CANCELLED = 9   /* the request was cancelled before it ran */
} rdct_status;

/* Which orthonormal transform a call applies (Sec. 2-3). */
typedef enum {
    RDCT_KIND_RDCT = 0, /* the proposed C_orth = S C0 (integer butterflies + folded scaling) */
    RDCT_KIND_DCT = 1   /* the exact 8-point DCT (FP32), the paper's comparison baseline */
} rdct_kind;

typedef void *rdct_stream; /* a cudaStream_t */

/* One 8-bit plane in device memory. */
typedef struct {
    const uint8_t *ptr; /* first pixel */
    int64_t pitch;      /* bytes between rows, >= w */
    int32_t w, h;       /* pixels; positive multiples of 8 */
} rdct_plane;

/* Reconstruction destination (device).  Either pointer may be NULL.
 * u8 has pitch `pitch` bytes; f32 has pitch `pitch_f32` floats. */
typedef struct {
    uint8_t *u8;
    float *f32;
    int64_t pitch;
    int64_t pitch_f32;
} rdct_out;

/* ---------------------------------------------------------------- basics */

RDCT_API const char *rdct_status_string(rdct_status s);
/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to cap bytes); returns its full length. */
RDCT_API size_t rdct_last_error(char *buf, size_t cap);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
RDCT_API int32_t rdct_version(void);
/* Blocks the host until all work on `stream` is done; reports async errors
 * (RDCT_ERR_CUDA).  Returns RDCT_ERR_TIMEOUT when a TMA-staged batch kernel
 * gave up waiting for a staged tile, or the tensor-core sweep pass for its
 * MMAs, since the last check (that warp or group stopped early, so that
 * launch's outputs and errors are incomplete); the counts are reset by the
 * check.  A staged tile that never arrived in time may still
 * land later in shared memory that another kernel then owns, so after a
 * timeout treat the results of every launch that ran at the same time as
 * suspect too. */
RDCT_API rdct_status rdct_sync(rdct_stream stream);

/* ------------------------------------------------------- the method's steps */

/* Forward transform Y = C0 A C0^T for every 8x8 block A of `src`
 * (Sec. 3 with T = C0; C0 from Sec. 2).  Y: int32, block-major,
 * (w/8)*(h/8)*64 values.  |Y| <= 16320, exact (additions only). */
RDCT_API rdct_status rdct_forward(const rdct_plane *src, int32_t *Y, rdct_stream stream);

/* Orthonormal forward coefficients in FP32, block-major [blocks][64]:
 * kind RDCT gives S Y S = C_orth A C_orth^T (Sec. 2), kind DCT gives C A C^T. */
RDCT_API rdct_status rdct_forward_f32(const rdct_plane *src, rdct_kind kind, float *Y, rdct_stream stream);

/* Compression (Sec. 2 "scaling merged into the quantization", Sec. 3 zonal
 * truncation): for each of `nblocks` blocks of int32 Y (block-major, 64
 * each), write the first r zigzag coefficients of S Y S as FP32, packed
 * [nblocks][r].  1 <= r <= 64. */
RDCT_API rdct_status rdct_compress(const int32_t *Y, int64_t nblocks, int32_t r, float *Yc, rdct_stream stream);

/* Inverse (Sec. 3 "inverse procedure", Sec. 2 orthogonality): from packed
 * [nbw*nbh][r] zigzag coefficients Yc, reconstruct Xhat = M^T Yhat M per
 * block (M = C_orth for kind RDCT, C for kind DCT; positions past r are
 * zero), writing FP32 and/or clamped rounded uint8 pixels into `out`
 * (an image of 8*nbw x 8*nbh pixels). */
RDCT_API rdct_status rdct_inverse(const float *Yc, int64_t nbw, int64_t nbh, int32_t r, rdct_kind kind,
                         const rdct_out *out, rdct_stream stream);

/* Quality (Sec. 3): MSE and PSNR = 10 log10(255^2 / MSE) of a reconstruction
 * against the reference plane.  rec->u8 is used when non-NULL, else
 * rec->f32.  mse and psnr are DEVICE pointers to one double each; PSNR is
 * +inf when MSE is 0.  Uses a small stream-ordered scratch allocation. */
RDCT_API rdct_status rdct_mse_psnr(const rdct_plane *ref, const rdct_out *rec, double *mse, double *psnr,
                          rdct_stream stream);

/* The other transforms the paper names, run through the same block experiment
 * (Sec. 3: Y = F A F^T, keep the first r zigzag coefficients, rebuild as
 * X = G Yhat G^T, score the squared error):
 *   ROUND       C_orth of Sec. 2 (the proposed transform; the general FP32
 *               kernel, a cross-check of the integer path);
 *   CEIL/FLOOR  the generalisations of the conclusion (Sec. 4): ceil(2C) or
 *               floor(2C) in place of [2C], orthogonalised the way Sec. 2
 *               orthogonalises C0 (the polar factor (T T^T)^(-1/2) T), G = F^T.
 *               floor(2C) has a zero first row, so it has no such factor and
 *               every call with FLOOR returns RDCT_ERR_ARG;
 *   SDCT        the signed DCT of the comparison in Sec. 3, sign(C)/sqrt(8)
 *               (the scaling of Table 2), rebuilt with its exact inverse
 *               (sign(C) is not orthogonal);
 *   SDCT_POLAR  sign(C) orthogonalised like C0, G = F^T.
 * The paper gives no compression inverse for these; the ones above are the
 * readings. */
typedef enum {
    RDCT_VARIANT_ROUND = 0,
    RDCT_VARIANT_CEIL = 1,
    RDCT_VARIANT_FLOOR = 2,
    RDCT_VARIANT_SDCT = 3,
    RDCT_VARIANT_SDCT_POLAR = 4
} rdct_variant;

/* The variant's forward matrix F and reconstruction matrix G, 64 doubles each,
 * row-major, written to HOST memory (computed on the host in double). */
RDCT_API rdct_status rdct_variant_matrices(rdct_variant v, double *F, double *G);

/* The whole experiment for one plane and one variant in one kernel (FP32
 * products, one thread per block): reconstruction to out (uint8
 * clamp(round(X)) and/or FP32 X, either may be NULL) and the plane's squared
 * error sum (X - A)^2 to *sse, a DEVICE double (8-byte aligned).  1 <= r <= 64.
 * Plane rules as for rdct_fused. */
RDCT_API rdct_status rdct_fused_variant(const rdct_plane *src, int32_t r, rdct_variant v, const rdct_out *out,
                                        double *sse, rdct_stream stream);

/* Spectral comparison of Sec. 2 (Fig. 2 and Table 2) for a variant's forward
 * matrix T (C_orth for ROUND, sign(C)/sqrt(8) for SDCT): D_m(w) =
 * |H_m(w; C) - H_m(w; T)|^2 with H_m(w; T) = sum_n t_{m,n} exp(-j n w), sampled
 * at w_i = i pi / (npoints - 1), i = 0 .. npoints-1, into D[m * npoints + i]
 * (HOST, 8 * npoints doubles, or NULL), and eps[m] = integral of D_m over
 * [0, pi] by the composite Simpson rule on that grid (HOST, 8 doubles).
 * npoints odd, 3 .. 2^24.  Host computation only (analysis, not the image
 * path). */
RDCT_API rdct_status rdct_spectral_error(rdct_variant v, int32_t npoints, double *D, double *eps);

/* Universal quality index of a reconstruction (Sec. 3 reports it beside PSNR
 * and MSE; its definition is in the work the paper cites): the mean over all
 * 8 x 8 windows (sliding by one pixel) of
 *   [2 s_xy / (s_x^2 + s_y^2)] * [2 mx my / (mx^2 + my^2)]
 * with window means, unbiased variances and covariance; a factor whose
 * denominator is zero counts as 1 (the paper gives no window size; 8 x 8 and
 * the flat-window rule are readings).  rec->u8 is used when non-NULL (exact
 * integer window sums), else rec->f32.  *q is a DEVICE double.  The plane
 * must be at least 8 x 8. */
RDCT_API rdct_status rdct_uqi(const rdct_plane *ref, const rdct_out *rec, double *q, rdct_stream stream);

/* The whole path in one kernel (Sec. 3): forward, keep r zigzag
 * coefficients with the S scaling, inverse, squared error.  `out` may be
 * NULL (error only).  *sse (DEVICE double) receives the sum over pixels of
 * (Xhat - A)^2 for the unrounded reconstruction; for kind RDCT it is exact
 * (integer arithmetic, 576 * SSE accumulated in 64 bits).  sse_u8 (DEVICE
 * double, 8-byte aligned, not the same slot as sse) may be NULL; otherwise it
 * receives the sum of (q - A)^2 for the 8-bit reconstruction
 * q = clamp(round(Xhat), 0, 255) that out->u8 holds (formed even when out or
 * out->u8 is NULL), exact for both kinds.  PSNR of the 8-bit image =
 * 10 log10(255^2 w h / sse_u8). */
RDCT_API rdct_status rdct_fused(const rdct_plane *src, int32_t r, rdct_kind kind, const rdct_out *out, double *sse,
                       double *sse_u8, rdct_stream stream);

/* The r sweep of Sec. 3 in one pass per plane: sse_by_r (DEVICE, [n][64]
 * doubles) receives, for each plane i and r = 1..64, the squared error of
 * the reconstruction keeping r coefficients, computed from the per-zigzag-
 * position energy of the orthonormal coefficients (Parseval: the transform
 * is orthogonal).  Exact for kind RDCT (integer transform and energies).  For
 * kind DCT the coefficients of 128 blocks at a time come from one tensor-core
 * product: the pixels exactly in FP16, C (x) C as the sum of two FP16 parts,
 * FP32 accumulation; FP32 sums per thread, FP64 sums per plane.  The
 * tensor-core pass waits for its MMAs with a bound; a wait that ran out is
 * reported by rdct_sync (RDCT_ERR_TIMEOUT: those planes' rows are
 * incomplete). */
RDCT_API rdct_status rdct_sweep(const rdct_plane *planes, int32_t n, rdct_kind kind, double *sse_by_r, rdct_stream stream);

/* rdct_sweep without any allocation.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they call in
 * (a framework that owns the whole device heap through its own allocator, a
 * real-time loop where an allocation could stall or synchronise the device, a
 * plug-in whose host process forbids device allocation).  Same arguments and
 * results as rdct_sweep; the per-call descriptor tables live in one fixed
 * device array inside the library (672 KiB, held on every GPU that
 * loads the library until the process exits) and are built on the device.
 * Limits: at most 2048 planes and 32768 chunks of 16 strips (about 1.07
 * Gpixel) per call, else RDCT_ERR_TOO_LARGE and nothing is enqueued.
 * The first call on a device looks up the array's device address (set-up,
 * once per device), so make it before any stream capture.  That address is
 * kept for the life of the process: do not reset the device
 * (cudaDeviceReset) while the library is loaded and this call is in use.  Every call shares
 * the array: calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. */
RDCT_API rdct_status rdct_sweep_noalloc(const rdct_plane *planes, int32_t n, rdct_kind kind, double *sse_by_r,
                                        rdct_stream stream);

/* ------------------------------------------------ batches of uneven planes */

/* One plane of a batch.  SSE is summed per image over its planes. */
typedef struct {
    rdct_plane src;
    uint8_t *dst;      /* uint8 reconstruction (device) or NULL */
    int64_t dst_pitch; /* bytes, >= src.w when dst != NULL */
    int32_t r;         /* 1..64 */
    int32_t image;     /* 0 <= image < nimages */
} rdct_job;

/* Launch shape of the persistent fused kernel. */
typedef struct {
    int32_t warps_per_cta;   /* 1..8 */
    int32_t ctas_per_sm;     /* grid = ctas_per_sm * SM count; 0 = as many as fit (at most 4 for
                                blocks_per_thread 2) */
    int32_t items_per_chunk; /* work items handed to a warp at a time (an item is one row of 32
                                lanes' blocks or block pairs) */
    int32_t blocks_per_thread; /* 2: two-block kernel (packed integer forward, f32x2 inverse), two
                                  vertically adjacent 8x8 blocks per thread, 4 warps per CTA;
                                  1: scalar kernel, one block per thread */
    int32_t staging;           /* blocks_per_thread 2 only.  0: TMA tile staging for the planes and r
                                  where it pays (16-byte aligned planes, r >= 16, nearly full
                                  32-column segments), per-thread copies elsewhere; 1: per-thread
                                  copies for every plane */
} rdct_tune;

typedef struct rdct_plan rdct_plan;

/* Build a plan over `njobs` planes: every plane is cut into work items
 * (runs of 32 column pairs, a pair being two vertically adjacent 8x8 blocks;
 * for planes that take TMA staging, 32-column segments of a row pair),
 * items are grouped into chunks ordered by r (with tune NULL and no cached
 * tune, each r's chunks are made small enough that the warps of its launch
 * get even shares), and the job and chunk tables
 * (and the planes' tensor maps) are uploaded to the device once.  tune may be
 * NULL (defaults / autotune cache).  All job pointers must stay valid while
 * the plan is used.  Errors: RDCT_ERR_ARG / RDCT_ERR_SHAPE naming the first
 * bad job, RDCT_ERR_OOM, RDCT_ERR_CUDA. */
RDCT_API rdct_status rdct_batch_plan_create(const rdct_job *jobs, int32_t njobs, int32_t nimages, const rdct_tune *tune,
                                   rdct_plan **plan);
/* Run the whole batch as one CUDA-graph launch: reset of the error slots,
 * one persistent kernel per r present (two where planes of that r take
 * different stagings), conversion of the slots to SSE.  The sequence is
 * captured on the first run with given (sse_per_image, sse_u8_per_image)
 * pointers and replayed afterwards on `stream`.  sse_per_image: DEVICE,
 * [nimages] doubles, 8-byte aligned, overwritten (unrounded reconstruction).
 * sse_u8_per_image: NULL, or another such array that receives each image's
 * squared error of its 8-bit reconstruction (exact). */
RDCT_API rdct_status rdct_batch_run(rdct_plan *plan, double *sse_per_image, double *sse_u8_per_image,
                                    rdct_stream stream);
/* Same work with one plain launch per plane (the baseline batching is
 * compared against). */
RDCT_API rdct_status rdct_batch_run_per_plane(rdct_plan *plan, double *sse_per_image, double *sse_u8_per_image,
                                              rdct_stream stream);
RDCT_API rdct_status rdct_batch_plan_get_tune(const rdct_plan *plan, rdct_tune *tune);
/* Kernels one rdct_batch_run launches (host): one per non-empty group of
 * chunks (an r, or a register class for the scalar kernel, and a staging
 * form) plus the conversion of the error slots.  RDCT_ERR_ARG on NULL. */
RDCT_API rdct_status rdct_batch_plan_kernels(const rdct_plan *plan, int32_t *kernels_per_run);
RDCT_API rdct_status rdct_batch_plan_destroy(rdct_plan *plan);

/* Time candidate launch shapes on this batch and return the fastest in
 * *best; the result is also kept in a per-process cache keyed by the batch's
 * shape class.  Candidates: the two-block kernel at 0 / 3 / 4 CTAs per SM,
 * 4..32 items per chunk, with and without TMA staging, and the scalar kernel.
 * Each is run once to capture and warm its graph, then timed over repeated
 * runs (CUDA events); a candidate whose runs spread by more than 5% is timed
 * again, and dropped if it stays that noisy.  The default shape is kept
 * unless a candidate's median beats it by more than 1%. */
RDCT_API rdct_status rdct_autotune(const rdct_job *jobs, int32_t njobs, int32_t nimages, rdct_tune *best, rdct_stream stream);
/* The autotune cache across processes.  Its keys name the GPU model (device
 * name, compute capability, SM count) and the batch's shape class, so a saved
 * cache applies to any device of that model.
 * rdct_autotune_cache_save writes every entry of this process's cache to
 * `path` (overwritten), one JSON object per line:
 *   {"key": "...", "warps_per_cta": 4, "ctas_per_sm": 4, "items_per_chunk": 32,
 *    "blocks_per_thread": 2, "staging": 0}
 * rdct_autotune_cache_load merges the lines of that exact form from `path`
 * into the cache (lines in any other form, or with an invalid launch shape,
 * are skipped) and reports how many it took in *loaded (may be NULL); plans
 * created with tune NULL then use them.  rdct_autotune_cache_clear empties the
 * cache.  Errors: RDCT_ERR_ARG (null path, unwritable file), RDCT_ERR_NOT_FOUND
 * (unreadable file). */
RDCT_API rdct_status rdct_autotune_cache_save(const char *path);
RDCT_API rdct_status rdct_autotune_cache_load(const char *path, int32_t *loaded);
RDCT_API rdct_status rdct_autotune_cache_clear(void);

/* -------------------------------------------- host-resident streaming path */

/* One plane in HOST memory (pinned or pageable) for the streaming calls. */
typedef struct {
    const uint8_t *src; /* host */
    uint8_t *dst;       /* host, may be NULL */
    int64_t pitch;      /* bytes, for both src and dst */
    int32_t w, h;
    int32_t r;
    int32_t image;
} rdct_host_job;

typedef struct rdct_pipeline rdct_pipeline;

/* A copy/compute pipeline with `device_budget_bytes` of staging memory split
 * into `depth` slots: host->device copies, kernels and device->host copies
 * of consecutive groups of planes overlap on separate streams. */
RDCT_API rdct_status rdct_pipeline_create(int64_t device_budget_bytes, int32_t depth, rdct_pipeline **pipe);
/* Process planes that live in host memory: copy in, run the fused path,
 * copy the uint8 reconstructions back, and write per-image SSE to the HOST
 * array sse_per_image[nimages] and, unless sse_u8_per_image is NULL, the
 * squared error of each image's 8-bit reconstruction to that HOST array.
 * Returns when everything is done. */
RDCT_API rdct_status rdct_pipeline_run(rdct_pipeline *pipe, const rdct_host_job *jobs, int32_t njobs, int32_t nimages,
                              double *sse_per_image, double *sse_u8_per_image);
RDCT_API rdct_status rdct_pipeline_destroy(rdct_pipeline *pipe);

/* How rdct_pipeline_run moves the planes:
 *   AUTO (default)  DIRECT when every plane (src and dst) is host memory the
 *                   device addresses with the same pointer: pinned memory, or
 *                   plain pageable memory on a device that reaches it through
 *                   the host's page tables (cudaDevAttrPageableMemoryAccess and
 *                   ...UsesHostPageTables, as on Grace-Blackwell nodes); else
 *                   STAGED;
 *   STAGED          host->device copies into device slots, kernels on the
 *                   slots, device->host copies, overlapped on three streams;
 *   DIRECT          the fused kernels read and write the host planes over the
 *                   host link (no staging); RDCT_ERR_ARG if a plane is not
 *                   such memory.
 * With pageable planes in DIRECT mode, the first device write to an output
 * page that the host has never touched faults the page in and is slow; output
 * buffers reused across runs (or touched once by the host) run at the link
 * rate. */
enum { RDCT_PIPELINE_AUTO = 0, RDCT_PIPELINE_STAGED = 1, RDCT_PIPELINE_DIRECT = 2 };
RDCT_API rdct_status rdct_pipeline_set_mode(rdct_pipeline *pipe, int32_t mode);

/* ----------------------------------------------------------------- serving */

typedef struct {
    int64_t device_budget_bytes; /* admission limit for resident request buffers */
    int32_t max_batch;           /* requests per launch, >= 1 */
    int32_t queue_capacity;      /* pending requests before submit returns BUSY */
    int32_t streams;             /* launches in flight, >= 1 */
    int32_t max_wait_us;         /* how long a lone request may wait for company */
} rdct_server_opts;

/* A request: an image of `planes` planes (1..4), all w x h, in host memory
 * (pinned or pageable): plane p starts at src + p * plane_stride
 * (plane_stride 0 means pitch * h), rows are `pitch` bytes apart; dst uses the
 * same layout.  Pinned planes move on the copy engines; pageable planes, on a
 * device that reaches pageable memory through the host page tables, are moved
 * by copy kernels (asynchronous, at the host-link rate), else by the driver's
 * staged copies. */
typedef struct {
    const uint8_t *src; /* host */
    uint8_t *dst;       /* host, receives the uint8 reconstruction (same layout), may be NULL */
    int64_t pitch;
    int64_t plane_stride;
    int32_t w, h, planes, r;
} rdct_request;

typedef struct {
    rdct_status status;
    double sse;        /* summed over planes, unrounded reconstruction */
    double mse, psnr;  /* over all samples of the image */
    double latency_us; /* submit -> completion */
    double sse_u8;     /* the same for the 8-bit reconstruction that is returned */
    double mse_u8, psnr_u8;
} rdct_result;

typedef struct {
    int64_t submitted, completed, rejected, batches;
    double p50_us, p99_us, mean_us;
    double gpixels_per_s; /* samples processed / busy wall time */
    int64_t peak_resident_bytes;
    double p999_us;
} rdct_server_stats;

typedef struct rdct_server rdct_server;

RDCT_API rdct_status rdct_server_create(const rdct_server_opts *opts, rdct_server **server);
/* Queue a request (host buffers must stay valid until it completes).
 * RDCT_ERR_BUSY if the queue is full, RDCT_ERR_TOO_LARGE if it can never fit
 * the budget. */
RDCT_API rdct_status rdct_server_submit(rdct_server *server, const rdct_request *req, uint64_t *ticket);
/* Wait up to timeout_us (negative = forever) for a ticket.  RDCT_ERR_TIMEOUT
 * leaves it pending; on success the ticket is retired. */
RDCT_API rdct_status rdct_server_wait(rdct_server *server, uint64_t ticket, int64_t timeout_us, rdct_result *result);
/* Non-blocking: RDCT_OK and the result if done, RDCT_ERR_BUSY if pending. */
RDCT_API rdct_status rdct_server_poll(rdct_server *server, uint64_t ticket, rdct_result *result);
/* Cancel a request that has not been admitted to the device yet. */
RDCT_API rdct_status rdct_server_cancel(rdct_server *server, uint64_t ticket);
RDCT_API rdct_status rdct_server_stats_get(rdct_server *server, rdct_server_stats *stats);
/* Drains outstanding work, then frees everything. */
RDCT_API rdct_status rdct_server_destroy(rdct_server *server);

/* Test hook for failure handling without a GPU fault: the next n buffer
 * admissions fail as if the device budget were exhausted; the affected
 * requests stay queued and are admitted once the failures are used up. */
RDCT_API rdct_status rdct_server_inject_alloc_failures(rdct_server *server, int32_t n);

/* ------------------------------------------- device-budget arena (host side) */

/* The first-fit sub-allocator the server uses to place request buffers in its
 * fixed device budget.  It manages offsets in [0, size) only (no memory of
 * its own), aligns every block to `align` bytes (a power of two) and merges
 * neighbouring free blocks on free. */
typedef struct rdct_arena rdct_arena;
RDCT_API rdct_status rdct_arena_create(int64_t size, int64_t align, rdct_arena **arena);
/* RDCT_ERR_OOM when no free block is large enough (nothing changes). */
RDCT_API rdct_status rdct_arena_alloc(rdct_arena *arena, int64_t bytes, int64_t *offset);
/* RDCT_ERR_NOT_FOUND when offset is not the start of a live block. */
RDCT_API rdct_status rdct_arena_free(rdct_arena *arena, int64_t offset);
RDCT_API int64_t rdct_arena_used(const rdct_arena *arena);
RDCT_API int64_t rdct_arena_largest_free(const rdct_arena *arena);
RDCT_API rdct_status rdct_arena_destroy(rdct_arena *arena);

#ifdef __cplusplus
}
#endif
#endif /* RDCT_H */
