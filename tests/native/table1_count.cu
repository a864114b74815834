// Counts the arithmetic of the 8-point butterflies the kernels use (Table 1 of
// the paper: the proposed transform needs 22 additions, no multiplications and
// no shifts).  c0_forward and c0t_inverse are instantiated on the host with a
// value type that counts every operation applied to it; the program prints the
// counts and checks, by applying the butterflies to the unit vectors, that
// they compute C0 x and C0^T x for the C0 printed in Sec. 2 (read from the
// fixture given on the command line).
#include <cstdio>
#include <cstdlib>

#include "rdct_device.cuh"

namespace {
long g_add = 0, g_mul = 0, g_shift = 0;

struct Counted {
    long v;
};
__host__ __device__ Counted operator+(Counted a, Counted b) {
#ifndef __CUDA_ARCH__
    ++g_add;
#endif
    return Counted{a.v + b.v};
}
__host__ __device__ Counted operator-(Counted a, Counted b) {
#ifndef __CUDA_ARCH__
    ++g_add;
#endif
    return Counted{a.v - b.v};
}
__host__ __device__ Counted operator-(Counted a) {
#ifndef __CUDA_ARCH__
    ++g_add;  // a negation is counted as an addition (it is a subtraction from zero)
#endif
    return Counted{-a.v};
}
__host__ __device__ Counted operator*(Counted a, Counted b) {
#ifndef __CUDA_ARCH__
    ++g_mul;
#endif
    return Counted{a.v * b.v};
}
__host__ __device__ Counted operator<<(Counted a, int s) {
#ifndef __CUDA_ARCH__
    ++g_shift;
#endif
    return Counted{a.v << s};
}
__host__ __device__ Counted operator>>(Counted a, int s) {
#ifndef __CUDA_ARCH__
    ++g_shift;
#endif
    return Counted{a.v >> s};
}
}  // namespace

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = std::fopen(argv[1], "r");
    if (!f) return 2;
    long C0[8][8];
    int got = 0;
    char line[512];
    while (got < 8 && std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        char *p = line, *e = nullptr;
        int n = 0;
        for (; n < 8; ++n) {
            const long v = std::strtol(p, &e, 10);
            if (e == p) break;
            C0[got][n] = v;
            p = e;
        }
        if (n == 8) ++got;
    }
    std::fclose(f);
    if (got != 8) return 2;

    // forward: one call on a general vector, counted
    Counted x[8], X[8];
    for (int n = 0; n < 8; ++n) x[n] = Counted{3 * n + 1};
    g_add = g_mul = g_shift = 0;
    rdct::c0_forward(x, X);
    std::printf("forward %ld %ld %ld\n", g_add, g_mul, g_shift);
    // inverse (all inputs present), counted
    Counted y[8];
    g_add = g_mul = g_shift = 0;
    rdct::c0t_inverse<0xFFu>(X, y);
    std::printf("inverse %ld %ld %ld\n", g_add, g_mul, g_shift);
    // the butterflies' responses to unit vectors against the printed matrix
    int bad = 0;
    for (int n = 0; n < 8; ++n) {
        Counted e[8], o[8], t[8];
        for (int k = 0; k < 8; ++k) e[k] = Counted{k == n ? 1 : 0};
        rdct::c0_forward(e, o);
        rdct::c0t_inverse<0xFFu>(e, t);
        for (int k = 0; k < 8; ++k) {
            bad += o[k].v != C0[k][n];   // column n of C0
            bad += t[k].v != C0[n][k];   // column n of C0^T = row n of C0
        }
    }
    std::printf("matrix %s\n", bad ? "mismatch" : "ok");
    return 0;
}
