// rdct_spectral.cu -- the spectral comparison of Sec. 2 (Fig. 2, Table 2), on
// the host: each row m of a transform matrix T is read as an FIR filter with
// transfer function H_m(w; T) = sum_n t_{m,n} exp(-j n w), its departure from
// the DCT's is D_m(w; T) = |H_m(w; C) - H_m(w; T)|^2, and the error energy is
// eps_m(T) = integral of D_m over [0, pi], evaluated numerically (composite
// Simpson rule on the sampling grid), as the paper does.
//
// T is the variant's forward matrix F: C_orth for the proposed transform and
// sign(C)/sqrt(8) for the signed DCT (the matrices Table 2 compares), the
// orthogonalised matrices for the other variants.  This is analysis, not part
// of the image path: a few thousand sample points, no device work.
#include <cmath>
#include <cstdint>

#include "rdct_internal.h"

using namespace rdct;

extern "C" rdct_status rdct_spectral_error(rdct_variant v, int32_t npoints, double *D, double *eps) {
    if (!eps) return set_error(RDCT_ERR_ARG, "rdct_spectral_error: null eps");
    if (npoints < 3 || npoints % 2 == 0 || npoints > (1 << 24))
        return set_error(RDCT_ERR_ARG, "rdct_spectral_error: npoints must be odd, 3 .. 2^24");
    double F[8][8], G[8][8];
    rdct_status st = variant_matrices(v, F, G);
    if (st) return st;
    const double pi = 3.14159265358979323846;
    double C[8][8];
    for (int k = 0; k < 8; ++k)
        for (int n = 0; n < 8; ++n) C[k][n] = (k == 0 ? std::sqrt(0.125) : 0.5) * std::cos(pi * (2 * n + 1) * k / 16.0);
    const double h = pi / (npoints - 1);
    for (int m = 0; m < 8; ++m) {
        double acc = 0.0;
        for (int32_t i = 0; i < npoints; ++i) {
            const double w = h * i;
            double re = 0.0, im = 0.0;  // H_m(w; C) - H_m(w; T)
            for (int n = 0; n < 8; ++n) {
                const double d = C[m][n] - F[m][n];
                re += d * std::cos(n * w);
                im -= d * std::sin(n * w);
            }
            const double dm = re * re + im * im;
            if (D) D[(int64_t)m * npoints + i] = dm;
            const double wt = (i == 0 || i == npoints - 1) ? 1.0 : (i % 2 ? 4.0 : 2.0);
            acc += wt * dm;
        }
        eps[m] = acc * h / 3.0;
    }
    return RDCT_OK;
}
