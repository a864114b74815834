// rdct_device.cuh -- device-side building blocks of the RDCT path (sm_103a).
//
// Everything here is derived from the structure of C0 = [2C] (Sec. 2 of Cintra
// & Bayer): even rows of C0 are symmetric and odd rows antisymmetric, which
// gives an 8-point butterfly with 22 additions (Table 1) for C0 and another 22
// for C0^T.  The orthogonalising scaling S (Sec. 2) is never applied as a
// multiplication inside the transform: C0 C0^T = diag(g) with
// g = (8,6,4,6,8,6,4,6), so S = diag(g)^(-1/2) and the whole scaled path
// C0^T S (mask . S Y S) S C0 equals C0^T (mask . W o Y) C0 / 576 with the
// integer weights W_ij = 576 / (g_i g_j) in {9,12,16,18,24,36}.
#pragma once
#include <cstdint>
#include <type_traits>

namespace rdct {

// ------------------------------------------------------------ constants

// Diagonal of C0 C0^T (row norms squared of C0: the number of non-zeros per row).
__host__ __device__ constexpr int gram(int i) {
    return (i == 0 || i == 4) ? 8 : ((i == 2 || i == 6) ? 4 : 6);
}
// 576 * d_i^2 * d_j^2 with d = diag(S): the integer form of the S Y S scaling.
__host__ __device__ constexpr int weight(int i, int j) { return 576 / (gram(i) * gram(j)); }
constexpr int kScale = 576;  // lcm of the g_i g_j products

// Zigzag rank of natural position (i, j): position of (i, j) in the JPEG scan
// (anti-diagonal s = i + j; odd s walk downward from the top row, even s walk
// upward from the left column).
__host__ __device__ constexpr int zz_rank(int i, int j) {
    int s = i + j;
    int before = 0;  // coefficients on the diagonals before s
    for (int t = 0; t < s; ++t) before += (t < 8) ? t + 1 : 15 - t;
    int lo = s > 7 ? s - 7 : 0;
    int hi = s < 7 ? s : 7;
    return (s & 1) ? before + (i - lo) : before + (hi - i);
}
// Anti-diagonal holding zigzag rank k (0..63).
__host__ __device__ constexpr int zz_diag_of_rank(int k) {
    int s = 0, before = 0;
    while (true) {
        int len = (s < 8) ? s + 1 : 15 - s;
        if (k < before + len) return s;
        before += len;
        ++s;
    }
}
// Natural index (row*8+col) of zigzag rank k.
__host__ __device__ constexpr int zz_pos(int k) {
    for (int p = 0; p < 64; ++p)
        if (zz_rank(p >> 3, p & 7) == k) return p;
    return -1;
}

// ------------------------------------------------------- compile-time loops

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// --------------------------------------------------- C0 forward butterfly

// X = C0 x for one 8-vector (22 additions).  V is any type with + and -
// (int32 here; exact since |X| <= 8 * max|x|).
template <typename V>
__host__ __device__ constexpr void c0_forward(const V x[8], V X[8]) {
    const V a0 = x[0] + x[7], a1 = x[1] + x[6], a2 = x[2] + x[5], a3 = x[3] + x[4];
    const V b0 = x[0] - x[7], b1 = x[1] - x[6], b2 = x[2] - x[5], b3 = x[3] - x[4];
    const V s03 = a0 + a3, s12 = a1 + a2;
    X[0] = s03 + s12;  // row 0: 1  1  1  1  1  1  1  1
    X[4] = s03 - s12;  // row 4: 1 -1 -1  1  1 -1 -1  1
    X[2] = a0 - a3;    // row 2: 1  0  0 -1 -1  0  0  1
    X[6] = a2 - a1;    // row 6: 0 -1  1  0  0  1 -1  0
    X[1] = b0 + b1 + b2;  // row 1: 1  1  1  0  0 -1 -1 -1
    X[3] = b0 - b2 - b3;  // row 3: 1  0 -1 -1  1  1  0 -1
    X[5] = b0 - b1 + b3;  // row 5: 1 -1  0  1 -1  0  1 -1
    X[7] = b2 - b1 - b3;  // row 7: 0 -1  1 -1  1 -1  1  0
}

// C0[k][n], read off the butterfly itself (its response to the unit vector e_n).
__host__ __device__ constexpr int c0_entry(int k, int n) {
    int x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int X[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    x[n] = 1;
    c0_forward(x, X);
    return X[k];
}
// Row k of C0 as four signed bytes per word: half 0 = columns 0..3, half 1 = 4..7
// (operands of a byte dot product with four packed pixels).
__host__ __device__ constexpr unsigned c0_row_word(int k, int half) {
    unsigned w = 0;
    for (int b = 0; b < 4; ++b) w |= ((unsigned)c0_entry(k, 4 * half + b) & 0xFFu) << (8 * b);
    return w;
}

// ---------------------------------------------- C0^T inverse butterfly (FP32)
//
// x = C0^T X for one 8-vector, in FP32, skipping inputs known at compile time
// to be zero (bit k of M set = X[k] may be non-zero).  All values on the RDCT
// path are integers below 2^24 in magnitude, so FP32 is exact here.

template <bool A, bool B, typename V>
__host__ __device__ __forceinline__ V padd(V a, V b) {
    if constexpr (A && B) return a + b;
    else if constexpr (A) return a;
    else if constexpr (B) return b;
    else return V{};
}
template <bool A, bool B, typename V>
__host__ __device__ __forceinline__ V psub(V a, V b) {
    if constexpr (A && B) return a - b;
    else if constexpr (A) return a;
    else if constexpr (B) return -b;
    else return V{};
}

// x = C0^T X for one 8-vector (22 additions at most), skipping inputs known
// at compile time to be zero (bit k of M set = X[k] may be non-zero).  V is
// float or a packed pair of floats; on the RDCT path every value is an
// integer (in some fixed unit) below 2^24 in magnitude, so it is exact.
// (Host-callable so that its operation count can be checked.)
template <unsigned M, typename V>
__host__ __device__ __forceinline__ void c0t_inverse(const V X[8], V x[8]) {
    constexpr bool p0 = M & 1u, p1 = (M >> 1) & 1u, p2 = (M >> 2) & 1u, p3 = (M >> 3) & 1u;
    constexpr bool p4 = (M >> 4) & 1u, p5 = (M >> 5) & 1u, p6 = (M >> 6) & 1u, p7 = (M >> 7) & 1u;
    // even half: columns n = 0..3 of rows 0, 2, 4, 6
    constexpr bool pp = p0 || p4;
    const V p = padd<p0, p4>(X[0], X[4]);
    const V q = psub<p0, p4>(X[0], X[4]);
    constexpr bool e0 = pp || p2, e1 = pp || p6;
    const V ea0 = padd<pp, p2>(p, X[2]);
    const V ea3 = psub<pp, p2>(p, X[2]);
    const V ea1 = psub<pp, p6>(q, X[6]);
    const V ea2 = padd<pp, p6>(q, X[6]);
    // odd half: columns n = 0..3 of rows 1, 3, 5, 7
    constexpr bool p13 = p1 || p3, p15 = p1 || p5, p35 = p3 || p5;
    const V t13 = padd<p1, p3>(X[1], X[3]);
    const V ob0 = padd<p13, p5>(t13, X[5]);   // X1 + X3 + X5
    const V t15 = psub<p1, p5>(X[1], X[5]);
    const V ob1 = psub<p15, p7>(t15, X[7]);   // X1 - X5 - X7
    const V t13m = psub<p1, p3>(X[1], X[3]);
    const V ob2 = padd<p13, p7>(t13m, X[7]);  // X1 - X3 + X7
    const V t53 = psub<p5, p3>(X[5], X[3]);
    const V ob3 = psub<p35, p7>(t53, X[7]);   // -X3 + X5 - X7
    constexpr bool o0 = p13 || p5, o1 = p15 || p7, o2 = p13 || p7, o3 = p35 || p7;
    constexpr bool e2 = e1, e3 = e0;
    x[0] = padd<e0, o0>(ea0, ob0);
    x[7] = psub<e0, o0>(ea0, ob0);
    x[1] = padd<e1, o1>(ea1, ob1);
    x[6] = psub<e1, o1>(ea1, ob1);
    x[2] = padd<e2, o2>(ea2, ob2);
    x[5] = psub<e2, o2>(ea2, ob2);
    x[3] = padd<e3, o3>(ea3, ob3);
    x[4] = psub<e3, o3>(ea3, ob3);
}

// Mask of rows i that hold retained coefficients in column j when every
// anti-diagonal up to D is (possibly) retained: i + j <= D.
__host__ __device__ constexpr unsigned col_mask(int D, int j) {
    int n = D - j + 1;
    if (n <= 0) return 0u;
    if (n >= 8) return 0xFFu;
    return (1u << n) - 1u;
}
// Columns that can hold retained coefficients: j <= D.
__host__ __device__ constexpr unsigned row_mask(int D) { return col_mask(D, 0); }

// First zigzag rank on anti-diagonal D and one past the last.
__host__ __device__ constexpr int diag_first_rank(int D) {
    int before = 0;
    for (int t = 0; t < D; ++t) before += (t < 8) ? t + 1 : 15 - t;
    return before;
}
__host__ __device__ constexpr int diag_end_rank(int D) { return diag_first_rank(D + 1); }

// The anti-diagonal class of r retained coefficients: the diagonal that holds
// rank r - 1.  Coefficients on earlier diagonals are always kept, those on
// later diagonals never, those on diagonal D are kept when their rank < r.
__host__ __device__ constexpr int diag_class(int r) { return zz_diag_of_rank(r - 1); }

// ----------------------------------------------------------- byte helpers

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int k) {
    return __byte_perm(w, 0u, 0x4440u + (unsigned)k);  // zero-extended byte k
}

// Rounding to 8 bits without conversion instructions.  A float times 2^-149
// lands in the subnormal range, where the representable values are the
// integer multiples of 2^-149: the multiplication rounds its exact product to
// the nearest integer (ties to even) and leaves that integer in the bit
// pattern; negative values carry the sign bit, so as int32 they are negative.
// cvt.pack.sat then clamps to [0, 255] while packing.
//
// q_from_576(e), e = 576 x an exact integer: e * 2^-149 is exact, and the
// multiplication by fl(1/576) (slightly above 1/576) rounds x to the nearest
// integer, exact halves upward.
__device__ __forceinline__ int q_from_576(float e) {
    return __float_as_int(__fmul_rn(__fmul_rn(e, 0x1p-149f), 1.0f / 576.0f));
}
// q_of(x): nearest integer of a plain FP32 value, ties to even.
__device__ __forceinline__ int q_of(float x) { return __float_as_int(__fmul_rn(x, 0x1p-149f)); }
// Four int32 values saturated to [0, 255], packed low byte first.
__device__ __forceinline__ uint32_t pack4_sat(int q0, int q1, int q2, int q3) {
    uint32_t hi, w;
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(hi) : "r"(q3), "r"(q2), "r"(0));
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(w) : "r"(q1), "r"(q0), "r"(hi));
    return w;
}

}  // namespace rdct
