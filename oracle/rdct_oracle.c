/*
 * rdct_oracle.c -- plain FP64 CPU oracle for the RDCT image-compression path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py may load this library.  The CUDA
 * library never links, includes or calls it, and it shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * What it computes (Cintra & Bayer, "A DCT Approximation for Image
 * Compression"):
 *   Sec. 2   C  = orthonormal 8-point DCT-II matrix ("standard DCT matrix").
 *   Sec. 2   C0 = [2C], [.] = Matlab round (half away from zero).
 *   Sec. 2   S  = sqrt((C0 C0^T)^-1), principal root; diagonal because
 *                 C0 C0^T is diagonal.  C_orth = S C0 is orthogonal.
 *   Sec. 3   each 8x8 block A -> M A M^T (M = C_orth, or C for the exact
 *                 DCT baseline); keep the first r coefficients of the standard
 *                 zigzag sequence, zero the rest; reconstruct with the inverse
 *                 (M orthogonal => inverse is M^T Yhat M); score with PSNR/MSE.
 *   Sec. 3-4 the same experiment for any forward matrix F and reconstruction
 *                 matrix G (rdct_ref_fused_general): the signed DCT compared
 *                 in Sec. 3 and the floor / ceiling generalisations that the
 *                 conclusion (Sec. 4) proposes; oracle.py builds the matrices.
 *   Sec. 3   UQI (the quality index cited there) on 8 x 8 sliding windows.
 *
 * Style: direct triple-loop 8x8 matrix products in double precision, in the
 * order the paper states them.  No butterflies, no fused scaling, no blocking.
 * The only liberty is an optional OpenMP loop over independent 8x8 blocks.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - zigzag: JPEG order, first step horizontal: (0,0),(0,1),(1,0),(2,0),...
 *     with (row = vertical frequency, column = horizontal frequency).
 *   - quality is measured on the unrounded reconstruction; the uint8 output is
 *     clamp(rint(x), 0, 255) with round-half-to-even (rint).
 *   - images whose sides are not multiples of 8 are rejected.
 *
 * Parity pins: every function here is pinned by tests that do not re-type its
 * formulas (printed C0 and S, Table 2, the 0.3922 scale, DC = block sum,
 * impulse responses, exact reconstruction at r = 64, Parseval, r = 1
 * equivalence with the DCT, scipy's orthonormal DCT for the exact baseline).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_SHAPE (-2)
#define ORACLE_ERR_NOT_DIAGONAL (-3)
#define ORACLE_ERR_NOT_INTEGER (-4)

/* ---------------------------------------------------------------- matrices */

/* Sec. 2: the standard (orthonormal) DCT-II matrix,
 * C[k][n] = a_k cos(pi (2n+1) k / 16), a_0 = sqrt(1/8), a_k = sqrt(2/8). */
void oracle_dct_matrix(double C[64]) {
    const double pi = acos(-1.0);
    for (int k = 0; k < 8; ++k) {
        double a = (k == 0) ? sqrt(1.0 / 8.0) : sqrt(2.0 / 8.0);
        for (int n = 0; n < 8; ++n)
            C[k * 8 + n] = a * cos(pi * (2.0 * n + 1.0) * k / 16.0);
    }
}

/* Sec. 2: Matlab's round(): nearest integer, halves away from zero. */
double oracle_matlab_round(double v) {
    double f = floor(fabs(v) + 0.5);
    return v < 0 ? -f : f;
}

/* Sec. 2: C0 = [2 C]. */
void oracle_round_off_matrix(double C0[64]) {
    double C[64];
    oracle_dct_matrix(C);
    for (int i = 0; i < 64; ++i) C0[i] = oracle_matlab_round(2.0 * C[i]);
}

/* out = a * b for 8x8 row-major matrices. */
static void matmul8(const double *a, const double *b, double *out) {
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += a[i * 8 + k] * b[k * 8 + j];
            out[i * 8 + j] = s;
        }
}

static void transpose8(const double *a, double *out) {
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) out[j * 8 + i] = a[i * 8 + j];
}

/* Sec. 2: S = sqrt((C0 C0^T)^-1) in the principal sense.  C0 C0^T is checked
 * to be diagonal with positive entries; for such a matrix the principal square
 * root of the inverse is the diagonal of 1/sqrt(entries).  Returns
 * ORACLE_ERR_NOT_DIAGONAL if the product has an off-diagonal non-zero (then
 * the principal root would need a general matrix function, which the paper's
 * matrix does not call for).  S is written as a full 8x8 matrix. */
int oracle_orthogonalizer(const double C0[64], double S[64]) {
    double C0t[64], P[64];
    transpose8(C0, C0t);
    matmul8(C0, C0t, P);
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            if (i != j && P[i * 8 + j] != 0.0) return ORACLE_ERR_NOT_DIAGONAL;
            if (i == j && !(P[i * 8 + j] > 0.0)) return ORACLE_ERR_NOT_DIAGONAL;
        }
    memset(S, 0, 64 * sizeof(double));
    for (int i = 0; i < 8; ++i) S[i * 8 + i] = sqrt(1.0 / P[i * 8 + i]);
    return ORACLE_OK;
}

/* Sec. 2: C_orth = S C0. */
int oracle_orth_matrix(double M[64]) {
    double C0[64], S[64];
    oracle_round_off_matrix(C0);
    int st = oracle_orthogonalizer(C0, S);
    if (st != ORACLE_OK) return st;
    matmul8(S, C0, M);
    return ORACLE_OK;
}

/* The orthonormal transform used for the 2-D experiment of Sec. 3:
 * kind 0 = C_orth (the proposed approximation), kind 1 = C (exact DCT). */
static int transform_matrix(int kind, double M[64]) {
    if (kind == 0) return oracle_orth_matrix(M);
    if (kind == 1) { oracle_dct_matrix(M); return ORACLE_OK; }
    return ORACLE_ERR_ARG;
}

/* Sec. 3 ("standard zigzag sequence"): walk the 15 anti-diagonals s = i + j;
 * odd s run from the top row downward (row increasing), even s run from the
 * left column upward (row decreasing), so the first step is horizontal.
 * zz[k] = row * 8 + col of the k-th coefficient in the sequence. */
void oracle_zigzag(int zz[64]) {
    int k = 0;
    for (int s = 0; s <= 14; ++s) {
        int lo = s > 7 ? s - 7 : 0;  /* smallest row on this diagonal */
        int hi = s < 7 ? s : 7;      /* largest row on this diagonal */
        if (s % 2 == 1) {
            for (int row = lo; row <= hi; ++row) zz[k++] = row * 8 + (s - row);
        } else {
            for (int row = hi; row >= lo; --row) zz[k++] = row * 8 + (s - row);
        }
    }
}

/* ------------------------------------------------------------ block helpers */

static int check_plane(const uint8_t *img, int64_t pitch, int32_t w, int32_t h) {
    if (!img || w <= 0 || h <= 0 || pitch < w) return ORACLE_ERR_ARG;
    if (w % 8 || h % 8) return ORACLE_ERR_SHAPE;
    return ORACLE_OK;
}

static void load_block(const uint8_t *img, int64_t pitch, int64_t by, int64_t bx, double A[64]) {
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) A[i * 8 + j] = (double)img[(by * 8 + i) * pitch + bx * 8 + j];
}

/* out = M A M^T (Sec. 3, the 2-D transform of a block). */
static void forward_block(const double *M, const double *A, double *out) {
    double Mt[64], tmp[64];
    transpose8(M, Mt);
    matmul8(M, A, tmp);
    matmul8(tmp, Mt, out);
}

/* out = M^T Y M (Sec. 3 "inverse procedure"; M orthogonal, Sec. 2). */
static void inverse_block(const double *M, const double *Y, double *out) {
    double Mt[64], tmp[64];
    transpose8(M, Mt);
    matmul8(Mt, Y, tmp);
    matmul8(tmp, M, out);
}

/* Zonal mask of Sec. 3: keep the first r zigzag coefficients, zero the rest. */
static void zonal_mask(const int zz[64], int r, const double *Y, double *out) {
    for (int i = 0; i < 64; ++i) out[i] = 0.0;
    for (int k = 0; k < r; ++k) out[zz[k]] = Y[zz[k]];
}

/* ----------------------------------------------------------- entry points */

/* Integer forward transform Y = C0 A C0^T (Sec. 3 with T = C0), block-major
 * output [by][bx][8][8] int32.  Computed in FP64 and converted only after
 * checking that every value is integral. */
int rdct_ref_forward(const uint8_t *img, int64_t pitch, int32_t w, int32_t h, int32_t *Y) {
    int st = check_plane(img, pitch, w, h);
    if (st) return st;
    double C0[64];
    oracle_round_off_matrix(C0);
    int64_t nbw = w / 8, nbh = h / 8;
    int bad = 0;
    for (int64_t by = 0; by < nbh; ++by)
        for (int64_t bx = 0; bx < nbw; ++bx) {
            double A[64], out[64];
            load_block(img, pitch, by, bx, A);
            forward_block(C0, A, out);
            int32_t *dst = Y + (by * nbw + bx) * 64;
            for (int i = 0; i < 64; ++i) {
                double rv = nearbyint(out[i]);
                if (fabs(out[i] - rv) > 1e-9) bad = 1;
                dst[i] = (int32_t)rv;
            }
        }
    return bad ? ORACLE_ERR_NOT_INTEGER : ORACLE_OK;
}

/* Orthonormal forward transform M A M^T in FP64, block-major [by][bx][64]
 * (kind 0: C_orth, kind 1: exact DCT C). */
int rdct_ref_forward_f64(const uint8_t *img, int64_t pitch, int32_t w, int32_t h, int32_t kind,
                         double *Y) {
    int st = check_plane(img, pitch, w, h);
    if (st) return st;
    double M[64];
    st = transform_matrix(kind, M);
    if (st) return st;
    int64_t nbw = w / 8, nbh = h / 8;
    for (int64_t by = 0; by < nbh; ++by)
        for (int64_t bx = 0; bx < nbw; ++bx) {
            double A[64];
            load_block(img, pitch, by, bx, A);
            forward_block(M, A, Y + (by * nbw + bx) * 64);
        }
    return ORACLE_OK;
}

/* Compression step (Sec. 2 "S merged into the quantization" + Sec. 3 zonal
 * truncation): for each block of integer coefficients Y = C0 A C0^T, form
 * S Y S (which equals C_orth A C_orth^T) and emit its first r zigzag
 * coefficients, packed [nblocks][r]. */
int rdct_ref_compress(const int32_t *Y, int64_t nblocks, int32_t r, double *Yc) {
    if (!Y || !Yc || nblocks < 0 || r < 1 || r > 64) return ORACLE_ERR_ARG;
    double C0[64], S[64];
    oracle_round_off_matrix(C0);
    int st = oracle_orthogonalizer(C0, S);
    if (st) return st;
    int zz[64];
    oracle_zigzag(zz);
    for (int64_t b = 0; b < nblocks; ++b) {
        double Yb[64], tmp[64], out[64];
        for (int i = 0; i < 64; ++i) Yb[i] = (double)Y[b * 64 + i];
        matmul8(S, Yb, tmp);
        matmul8(tmp, S, out);
        for (int k = 0; k < r; ++k) Yc[b * r + k] = out[zz[k]];
    }
    return ORACLE_OK;
}

/* Inverse (Sec. 3): unpack r zigzag coefficients per block into an 8x8 block
 * with zeros elsewhere, reconstruct M^T Yhat M, write FP64 pixels (row-major,
 * pitch xpitch elements).  Blocks are in raster order, nbw x nbh. */
int rdct_ref_inverse(const double *Yc, int64_t nbw, int64_t nbh, int32_t r, int32_t kind,
                     double *X, int64_t xpitch) {
    if (!Yc || !X || nbw < 0 || nbh < 0 || r < 1 || r > 64 || xpitch < nbw * 8) return ORACLE_ERR_ARG;
    double M[64];
    int st = transform_matrix(kind, M);
    if (st) return st;
    int zz[64];
    oracle_zigzag(zz);
    for (int64_t by = 0; by < nbh; ++by)
        for (int64_t bx = 0; bx < nbw; ++bx) {
            const double *src = Yc + (by * nbw + bx) * r;
            double Yh[64], out[64];
            for (int i = 0; i < 64; ++i) Yh[i] = 0.0;
            for (int k = 0; k < r; ++k) Yh[zz[k]] = src[k];
            inverse_block(M, Yh, out);
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) X[(by * 8 + i) * xpitch + bx * 8 + j] = out[i * 8 + j];
        }
    return ORACLE_OK;
}

/* uint8 version of a reconstruction: clamp(rint(x), 0, 255). */
static uint8_t to_u8(double x) {
    double v = nearbyint(x);
    if (v < 0) v = 0;
    if (v > 255) v = 255;
    return (uint8_t)v;
}

/* The whole experiment of Sec. 3 for one plane at one r:
 * forward, zonal truncation, inverse, squared error.
 *   xhat  (nullable) FP64 reconstruction, row-major, pitch w
 *   u8    (nullable) clamp(rint(xhat)), row-major, pitch w
 *   sse   sum over pixels of (xhat - a)^2 (unrounded reconstruction)
 *   sse_u8 (nullable) sum of (u8 - a)^2
 * nthreads <= 0 uses the OpenMP default; blocks are independent. */
int rdct_ref_fused(const uint8_t *img, int64_t pitch, int32_t w, int32_t h, int32_t r, int32_t kind,
                   double *xhat, uint8_t *u8, double *sse, double *sse_u8, int32_t nthreads) {
    int st = check_plane(img, pitch, w, h);
    if (st) return st;
    if (r < 1 || r > 64 || !sse) return ORACLE_ERR_ARG;
    double M[64];
    st = transform_matrix(kind, M);
    if (st) return st;
    int zz[64];
    oracle_zigzag(zz);
    int64_t nbw = w / 8, nbh = h / 8;
    double acc = 0.0, acc_u8 = 0.0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) reduction(+ : acc, acc_u8) num_threads(nt)
#endif
    for (int64_t by = 0; by < nbh; ++by) {
        for (int64_t bx = 0; bx < nbw; ++bx) {
            double A[64], Y[64], Yh[64], X[64];
            load_block(img, pitch, by, bx, A);
            forward_block(M, A, Y);
            zonal_mask(zz, r, Y, Yh);
            inverse_block(M, Yh, X);
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) {
                    double x = X[i * 8 + j], a = A[i * 8 + j];
                    int64_t o = (by * 8 + i) * (int64_t)w + bx * 8 + j;
                    acc += (x - a) * (x - a);
                    uint8_t q = to_u8(x);
                    acc_u8 += ((double)q - a) * ((double)q - a);
                    if (xhat) xhat[o] = x;
                    if (u8) u8[o] = q;
                }
        }
    }
    (void)nthreads;
    *sse = acc;
    if (sse_u8) *sse_u8 = acc_u8;
    return ORACLE_OK;
}

/* The Sec. 3 experiment with any pair of 8x8 matrices: each block A goes to
 * Y = F A F^T, keeps the first r zigzag coefficients, and is rebuilt as
 * X = G Yhat G^T.  This serves the generalisations of the conclusion (C0
 * built with floor or ceiling instead of round-off, orthogonalised by the
 * polar factor of Sec. 2) and the signed DCT compared in Sec. 3, whose
 * matrices the caller supplies (row-major).  Same outputs as rdct_ref_fused.
 * Pinned by the Kronecker form vec(F A F^T) = (F kron F) vec(A) on small
 * planes, exact reconstruction at r = 64 and agreement with rdct_ref_fused
 * for C_orth. */
int rdct_ref_fused_general(const uint8_t *img, int64_t pitch, int32_t w, int32_t h, int32_t r, const double *F,
                           const double *G, double *xhat, uint8_t *u8, double *sse, double *sse_u8,
                           int32_t nthreads) {
    int st = check_plane(img, pitch, w, h);
    if (st) return st;
    if (r < 1 || r > 64 || !sse || !F || !G) return ORACLE_ERR_ARG;
    double Ft[64], Gt[64];
    transpose8(F, Ft);
    transpose8(G, Gt);
    int zz[64];
    oracle_zigzag(zz);
    int64_t nbw = w / 8, nbh = h / 8;
    double acc = 0.0, acc_u8 = 0.0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) reduction(+ : acc, acc_u8) num_threads(nt)
#endif
    for (int64_t by = 0; by < nbh; ++by) {
        for (int64_t bx = 0; bx < nbw; ++bx) {
            double A[64], tmp[64], Y[64], Yh[64], X[64];
            load_block(img, pitch, by, bx, A);
            matmul8(F, A, tmp);
            matmul8(tmp, Ft, Y);
            zonal_mask(zz, r, Y, Yh);
            matmul8(G, Yh, tmp);
            matmul8(tmp, Gt, X);
            for (int i = 0; i < 8; ++i)
                for (int j = 0; j < 8; ++j) {
                    double x = X[i * 8 + j], a = A[i * 8 + j];
                    int64_t o = (by * 8 + i) * (int64_t)w + bx * 8 + j;
                    acc += (x - a) * (x - a);
                    uint8_t q = to_u8(x);
                    acc_u8 += ((double)q - a) * ((double)q - a);
                    if (xhat) xhat[o] = x;
                    if (u8) u8[o] = q;
                }
        }
    }
    (void)nthreads;
    *sse = acc;
    if (sse_u8) *sse_u8 = acc_u8;
    return ORACLE_OK;
}

/* Sweep of Sec. 3 over r = 1..64 for one plane: sse_by_r[r-1] is the squared
 * error of the reconstruction that keeps r coefficients, each obtained by a
 * direct inverse (no energy shortcut). */
int rdct_ref_sweep(const uint8_t *img, int64_t pitch, int32_t w, int32_t h, int32_t kind,
                   double *sse_by_r, int32_t nthreads) {
    int st = check_plane(img, pitch, w, h);
    if (st) return st;
    if (!sse_by_r) return ORACLE_ERR_ARG;
    for (int r = 1; r <= 64; ++r) {
        st = rdct_ref_fused(img, pitch, w, h, r, kind, NULL, NULL, &sse_by_r[r - 1], NULL, nthreads);
        if (st) return st;
    }
    return ORACLE_OK;
}

/* Sum of squared differences between a uint8 reference plane and a
 * reconstruction given either as uint8 (rec_u8) or FP64 (rec_f64), both
 * row-major with their own pitches (elements). */
int rdct_ref_sse(const uint8_t *ref, int64_t pitch, int32_t w, int32_t h, const uint8_t *rec_u8,
                 const double *rec_f64, int64_t rec_pitch, double *sse) {
    if (!ref || !sse || (!rec_u8 && !rec_f64) || w <= 0 || h <= 0 || pitch < w || rec_pitch < w)
        return ORACLE_ERR_ARG;
    double acc = 0.0;
    for (int64_t y = 0; y < h; ++y)
        for (int64_t x = 0; x < w; ++x) {
            double a = ref[y * pitch + x];
            double b = rec_u8 ? (double)rec_u8[y * rec_pitch + x] : rec_f64[y * rec_pitch + x];
            acc += (b - a) * (b - a);
        }
    *sse = acc;
    return ORACLE_OK;
}

/* Universal quality index (the UQI of Sec. 3, defined in the work it cites,
 * Wang & Bovik 2002): for every B x B window (sliding by one pixel) of the
 * reference x and the reconstruction y,
 *   Q = 4 s_xy mx my / ((s_x^2 + s_y^2)(mx^2 + my^2))
 *     = [2 s_xy / (s_x^2 + s_y^2)] * [2 mx my / (mx^2 + my^2)]
 * with sample means mx, my, unbiased variances s_x^2, s_y^2 and covariance
 * s_xy; the index is the mean of Q over all windows.  Reading for flat
 * windows: a factor whose denominator is zero is taken as 1 (its limit for
 * equal windows).  Computed directly per window in double precision. */
int rdct_ref_uqi(const uint8_t *ref, int64_t pitch, int32_t w, int32_t h, const uint8_t *rec_u8,
                 const double *rec_f64, int64_t rec_pitch, int32_t B, double *q) {
    if (!ref || !q || (!rec_u8 && !rec_f64) || B < 2 || w < B || h < B || pitch < w || rec_pitch < w)
        return ORACLE_ERR_ARG;
    const double n = (double)B * B;
    double total = 0.0;
    int64_t count = 0;
    for (int64_t y0 = 0; y0 + B <= h; ++y0)
        for (int64_t x0 = 0; x0 + B <= w; ++x0) {
            double mx = 0, my = 0;
            for (int i = 0; i < B; ++i)
                for (int j = 0; j < B; ++j) {
                    mx += ref[(y0 + i) * pitch + x0 + j];
                    my += rec_u8 ? (double)rec_u8[(y0 + i) * rec_pitch + x0 + j]
                                 : rec_f64[(y0 + i) * rec_pitch + x0 + j];
                }
            mx /= n;
            my /= n;
            double vx = 0, vy = 0, cxy = 0;
            for (int i = 0; i < B; ++i)
                for (int j = 0; j < B; ++j) {
                    const double a = ref[(y0 + i) * pitch + x0 + j] - mx;
                    const double b = (rec_u8 ? (double)rec_u8[(y0 + i) * rec_pitch + x0 + j]
                                             : rec_f64[(y0 + i) * rec_pitch + x0 + j]) - my;
                    vx += a * a;
                    vy += b * b;
                    cxy += a * b;
                }
            vx /= n - 1;
            vy /= n - 1;
            cxy /= n - 1;
            const double d1 = vx + vy, d2 = mx * mx + my * my;
            const double f1 = d1 == 0.0 ? 1.0 : 2.0 * cxy / d1;
            const double f2 = d2 == 0.0 ? 1.0 : 2.0 * mx * my / d2;
            total += f1 * f2;
            ++count;
        }
    *q = total / (double)count;
    return ORACLE_OK;
}

int rdct_ref_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
