// rdct_variant.cu -- matrices and entry points of the other transforms the
// paper names: the signed DCT of its comparison (Sec. 3) and the floor /
// ceiling generalisations of C0 = [2C] proposed in its conclusion (Sec. 4).
//
// Construction (host, double precision):
//   C        orthonormal 8-point DCT-II, C[k][n] = a_k cos(pi (2n+1) k / 16).
//   T        round-off (half away from zero), ceiling or floor of 2C, or
//            sign(C) for the signed DCT.
//   polar    F = (T T^T)^(-1/2) T, the orthogonal polar factor of T (the
//            orthogonalisation Sec. 2 applies to C0), with the inverse square
//            root taken through a cyclic Jacobi eigendecomposition of the
//            symmetric positive definite T T^T; G = F^T.
//   SDCT     F = sign(C) / sqrt(8) (the scaling Table 2 uses) and G = F^-1
//            (Gauss-Jordan with partial pivoting), since sign(C) is not
//            orthogonal.
// floor(2C) has a zero first row (2 a_0 = 1/sqrt(2) < 1), so T T^T is singular
// and the variant is refused.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "rdct_internal.h"

namespace rdct {
namespace {

constexpr double kPi = 3.14159265358979323846;

void dct_matrix(double C[8][8]) {
    for (int k = 0; k < 8; ++k)
        for (int n = 0; n < 8; ++n)
            C[k][n] = (k == 0 ? std::sqrt(0.125) : 0.5) * std::cos(kPi * (2 * n + 1) * k / 16.0);
}

void matmul(const double A[8][8], const double B[8][8], double out[8][8]) {
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += A[i][k] * B[k][j];
            out[i][j] = s;
        }
}

// Cyclic Jacobi: rotations J(p, q) with J_pp = J_qq = c, J_pq = s, J_qp = -s
// zero the (p, q) entry of J^T A J when t = s / c solves
// t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq) (smaller root).
// On return A = V diag(lam) V^T.
bool sym_eig(const double A_in[8][8], double V[8][8], double lam[8]) {
    double A[8][8];
    std::memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, scale = 0.0;
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j) (i == j ? scale : off) += A[i][j] * A[i][j];
        if (off <= 1e-30 * scale) {
            for (int i = 0; i < 8; ++i) lam[i] = A[i][i];
            return true;
        }
        for (int p = 0; p < 7; ++p)
            for (int q = p + 1; q < 8; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                // A <- A J (columns p, q), then A <- J^T A (rows p, q); V <- V J.
                for (int k = 0; k < 8; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 8; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 8; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    return false;
}

// Gauss-Jordan elimination with partial pivoting; false if singular.
bool invert(const double A_in[8][8], double inv[8][8]) {
    double a[8][16];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 16; ++j) a[i][j] = j < 8 ? A_in[i][j] : (j - 8 == i ? 1.0 : 0.0);
    for (int col = 0; col < 8; ++col) {
        int piv = col;
        for (int i = col + 1; i < 8; ++i)
            if (std::fabs(a[i][col]) > std::fabs(a[piv][col])) piv = i;
        if (std::fabs(a[piv][col]) < 1e-12) return false;
        if (piv != col)
            for (int j = 0; j < 16; ++j) std::swap(a[piv][j], a[col][j]);
        const double d = a[col][col];
        for (int j = 0; j < 16; ++j) a[col][j] /= d;
        for (int i = 0; i < 8; ++i) {
            if (i == col || a[i][col] == 0.0) continue;
            const double f = a[i][col];
            for (int j = 0; j < 16; ++j) a[i][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) inv[i][j] = a[i][j + 8];
    return true;
}

double max_dev_identity(const double P[8][8]) {
    double m = 0.0;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) m = std::fmax(m, std::fabs(P[i][j] - (i == j ? 1.0 : 0.0)));
    return m;
}

}  // namespace

rdct_status variant_matrices(rdct_variant v, double F[8][8], double G[8][8]) {
    double C[8][8], T[8][8];
    dct_matrix(C);
    for (int k = 0; k < 8; ++k)
        for (int n = 0; n < 8; ++n) {
            const double x = 2.0 * C[k][n];
            switch (v) {
                case RDCT_VARIANT_ROUND: T[k][n] = std::round(x); break;  // half away from zero
                case RDCT_VARIANT_CEIL: T[k][n] = std::ceil(x); break;
                case RDCT_VARIANT_FLOOR: T[k][n] = std::floor(x); break;
                case RDCT_VARIANT_SDCT:
                case RDCT_VARIANT_SDCT_POLAR: T[k][n] = C[k][n] > 0 ? 1.0 : -1.0; break;
                default: return set_error(RDCT_ERR_ARG, "rdct_variant: unknown variant");
            }
        }
    if (v == RDCT_VARIANT_SDCT) {
        for (int k = 0; k < 8; ++k)
            for (int n = 0; n < 8; ++n) F[k][n] = T[k][n] / std::sqrt(8.0);
        if (!invert(F, G)) return set_error(RDCT_ERR_ARG, "rdct_variant: signed DCT matrix is singular");
        double P[8][8];
        matmul(G, F, P);
        if (max_dev_identity(P) > 1e-12) return set_error(RDCT_ERR_ARG, "rdct_variant: inverse check failed");
        return RDCT_OK;
    }
    double Tt[8][8], gram[8][8], V[8][8], lam[8];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) Tt[i][j] = T[j][i];
    matmul(T, Tt, gram);
    if (!sym_eig(gram, V, lam)) return set_error(RDCT_ERR_ARG, "rdct_variant: eigendecomposition did not converge");
    double lmax = 0.0, lmin = INFINITY;
    for (int i = 0; i < 8; ++i) {
        lmax = std::fmax(lmax, lam[i]);
        lmin = std::fmin(lmin, lam[i]);
    }
    if (!(lmin > 1e-9 * lmax))
        return set_error(RDCT_ERR_ARG, "rdct_variant: T T^T is singular (floor(2C) has a zero first row)");
    double S[8][8];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += V[i][k] * V[j][k] / std::sqrt(lam[k]);
            S[i][j] = s;
        }
    matmul(S, T, F);
    double Ft[8][8], P[8][8];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) G[i][j] = Ft[i][j] = F[j][i];
    matmul(F, Ft, P);
    if (max_dev_identity(P) > 1e-12) return set_error(RDCT_ERR_ARG, "rdct_variant: polar factor not orthogonal");
    return RDCT_OK;
}

namespace {

cudaError_t launch_variant(int d, const JobDesc &job, const MatConsts &M, double *acc, cudaStream_t s) {
    switch (d) {
        case 0: return launch_variant_d<0>(job, M, acc, s);
        case 1: return launch_variant_d<1>(job, M, acc, s);
        case 2: return launch_variant_d<2>(job, M, acc, s);
        case 3: return launch_variant_d<3>(job, M, acc, s);
        case 4: return launch_variant_d<4>(job, M, acc, s);
        case 5: return launch_variant_d<5>(job, M, acc, s);
        case 6: return launch_variant_d<6>(job, M, acc, s);
        case 7: return launch_variant_d<7>(job, M, acc, s);
        case 8: return launch_variant_d<8>(job, M, acc, s);
        case 9: return launch_variant_d<9>(job, M, acc, s);
        case 10: return launch_variant_d<10>(job, M, acc, s);
        case 11: return launch_variant_d<11>(job, M, acc, s);
        case 12: return launch_variant_d<12>(job, M, acc, s);
        case 13: return launch_variant_d<13>(job, M, acc, s);
        default: return launch_variant_d<14>(job, M, acc, s);
    }
}

}  // namespace
}  // namespace rdct

using namespace rdct;

extern "C" rdct_status rdct_variant_matrices(rdct_variant v, double *F, double *G) {
    if (!F || !G) return set_error(RDCT_ERR_ARG, "rdct_variant_matrices: null output");
    double f[8][8], g[8][8];
    rdct_status st = variant_matrices(v, f, g);
    if (st) return st;
    std::memcpy(F, f, sizeof(f));
    std::memcpy(G, g, sizeof(g));
    return RDCT_OK;
}

extern "C" rdct_status rdct_fused_variant(const rdct_plane *src, int32_t r, rdct_variant v, const rdct_out *out,
                                          double *sse, rdct_stream stream) {
    rdct_status st = validate_plane(src, "rdct_fused_variant");
    if (st) return st;
    if (r < 1 || r > 64) return set_error(RDCT_ERR_ARG, "rdct_fused_variant: r must be in 1..64");
    if (!sse) return set_error(RDCT_ERR_ARG, "rdct_fused_variant: null sse");
    if (reinterpret_cast<uintptr_t>(sse) % 8) return set_error(RDCT_ERR_ARG, "rdct_fused_variant: misaligned sse");
    if (out && out->u8 && out->pitch < src->w) return set_error(RDCT_ERR_SHAPE, "out: u8 pitch smaller than width");
    if (out && out->f32 && out->pitch_f32 < src->w)
        return set_error(RDCT_ERR_SHAPE, "out: f32 pitch smaller than width");
    double f[8][8], g[8][8];
    st = variant_matrices(v, f, g);
    if (st) return st;
    MatConsts M;
    for (int i = 0; i < 64; ++i) {
        M.f[i] = (float)f[i / 8][i % 8];
        M.g[i] = (float)g[i / 8][i % 8];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const JobDesc job = make_job(*src, out ? out->u8 : nullptr, out ? out->pitch : 0, out ? out->f32 : nullptr,
                                 out ? out->pitch_f32 : 0, r, 0, 1);
    RDCT_CUDA_TRY(cudaMemsetAsync(sse, 0, sizeof(double), s));
    RDCT_CUDA_TRY(launch_variant(diag_class_host(r), job, M, sse, s));
    return RDCT_OK;
}
