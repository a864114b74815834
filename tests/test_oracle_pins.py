"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types an oracle formula: each compares the oracle with
a printed value of the paper (tests/golden/), a closed form, an invariant, a
library routine for a special case (scipy's orthonormal DCT), or brute force
on tiny inputs built from the printed matrix.  A dropped term, a wrong sign, a
transposed operand or an off-by-one in the zonal mask fails at least one.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import oracle as orc
from paper_1402_6034_gb300 import synth
from tests.conftest import load_golden

FULL_DIAGONALS = [1, 3, 6, 10, 15, 21, 28, 36, 43, 49, 54, 58, 61, 63, 64]


# ------------------------------------------------------------------ matrices

def test_round_off_matrix_matches_printed(golden_c0):
    """Sec. 2: [2C] equals the printed C0 entry by entry."""
    np.testing.assert_array_equal(orc.round_off_matrix(), golden_c0)


def test_matlab_round_is_half_away_from_zero():
    """Sec. 2: Matlab's round sends halves away from zero."""
    for v, e in [(0.5, 1), (-0.5, -1), (1.5, 2), (2.5, 3), (-2.5, -3), (0.49, 0), (-0.51, -1)]:
        assert orc.matlab_round(v) == e


def test_no_tie_in_2c():
    """Sec. 2: no entry of 2C sits near a half, so the tie rule cannot change C0."""
    frac = np.abs(2 * orc.dct_matrix()) % 1.0
    assert np.min(np.abs(frac - 0.5)) > 0.05


def test_c0_gram_is_diagonal(golden_c0):
    """Sec. 2: C0 C0^T is diagonal, diag(8,6,4,6,8,6,4,6), so S is diagonal."""
    g = golden_c0 @ golden_c0.T
    np.testing.assert_array_equal(g, np.diag([8, 6, 4, 6, 8, 6, 4, 6]))


def test_orthogonalizer_matches_printed_s(golden_c0):
    """Sec. 2: S = sqrt((C0 C0^T)^-1) equals the printed diagonal."""
    d2 = np.array([float(r[0]) for r in load_golden("s_diag.txt")])
    S = orc.orthogonalizer(golden_c0)
    np.testing.assert_allclose(S, np.diag(1.0 / np.sqrt(d2)), rtol=0, atol=1e-15)


def test_orthogonalizer_rejects_non_diagonal_gram():
    """The diagonal closed form is only used when C0 C0^T is diagonal."""
    m = np.eye(8)
    m[0, 1] = 1.0
    with pytest.raises(RuntimeError):
        orc.orthogonalizer(m)


def test_orth_matrix_is_orthogonal():
    """Sec. 2: C_orth = S C0 is orthogonal."""
    M = orc.orth_matrix()
    np.testing.assert_allclose(M @ M.T, np.eye(8), atol=1e-15)
    np.testing.assert_allclose(M.T @ M, np.eye(8), atol=1e-15)


def test_dct_matrix_matches_scipy():
    """C is the orthonormal DCT-II: C x equals scipy's dct(x, norm='ortho')."""
    C = orc.dct_matrix()
    eye = np.eye(8)
    ref = scipy.fft.dct(eye, type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(C, ref, atol=1e-15)


def test_frobenius_optimal_scale():
    """Sec. 2: argmin_a ||a C0 - C||_F rounds to the printed 0.3922."""
    C, C0 = orc.dct_matrix(), orc.round_off_matrix()
    a = np.sum(C * C0) / np.sum(C0 * C0)
    printed = float(load_golden("scale_0p3922.txt")[0][0])
    assert round(a, 4) == printed
    # the minimiser really is a minimum of the Frobenius distance
    f = lambda s: np.linalg.norm(s * C0 - C)
    assert f(a) < f(a - 1e-3) and f(a) < f(a + 1e-3)


def test_table2_error_energy():
    """Sec. 2, Table 2: eps_m of the proposed C_orth and of the SDCT (sign(C)/sqrt8)."""
    rows = load_golden("table2.txt")
    eps_p = orc.error_energy(orc.orth_matrix())
    eps_s = orc.error_energy(orc.sdct_matrix())
    for row in rows[:-1]:
        m = int(row[0])
        assert round(eps_s[m], 2) == pytest.approx(float(row[1]), abs=1e-9), (m, eps_s[m])
        assert round(eps_p[m], 2) == pytest.approx(float(row[2]), abs=1e-9), (m, eps_p[m])
    sel = [1, 2, 3, 5, 6, 7]
    assert round(eps_s[sel].sum(), 2) == pytest.approx(float(rows[-1][1]))
    assert round(eps_p[sel].sum(), 2) == pytest.approx(float(rows[-1][2]))
    # Sec. 2: rows 0 and 4 of the approximation coincide with the DCT's
    assert eps_p[0] < 1e-20 and eps_p[4] < 1e-20


def test_error_energy_quadrature_against_closed_form():
    """The Simpson quadrature is exact to 1e-12 on a case with a closed form:
    for real taps c, integral_0^pi |sum_n c_n e^{-jnw}|^2 dw = pi * ||c||^2."""
    rng = np.random.default_rng(3)
    T = rng.standard_normal((8, 8))
    C = orc.dct_matrix()
    eps = orc.error_energy(T)
    np.testing.assert_allclose(eps, np.pi * np.sum((C - T) ** 2, axis=1), rtol=1e-12)


# -------------------------------------------------------------------- zigzag

def test_zigzag_matches_jpeg_scan():
    """Reading of Sec. 3's 'standard zigzag sequence': the JPEG scan order."""
    table = np.array([int(v) for row in load_golden("zigzag_jpeg.txt") for v in row])
    np.testing.assert_array_equal(orc.zigzag(), table)


def test_zigzag_structure():
    """A permutation whose rank grows with the anti-diagonal i + j."""
    zz = orc.zigzag()
    assert sorted(zz.tolist()) == list(range(64))
    diag = (zz // 8) + (zz % 8)
    assert np.all(np.diff(diag) >= 0)


# ------------------------------------------------------------------- forward

def test_forward_dc_is_block_sum():
    """Row 0 of C0 is all ones (Sec. 2), so Y[0][0] is the sum of the block."""
    img = synth.random_bytes((32, 48), seed=1)
    Y = orc.forward(img)
    sums = img.reshape(4, 8, 6, 8).sum(axis=(1, 3))
    np.testing.assert_array_equal(Y[:, :, 0, 0], sums)


def test_forward_impulses(golden_c0):
    """An impulse of height v at (i, j) transforms to v * C0[:, i] C0[:, j]^T."""
    for v in (1, 255):
        for i in range(8):
            for j in range(8):
                img = np.zeros((8, 8), np.uint8)
                img[i, j] = v
                Y = orc.forward(img)[0, 0]
                np.testing.assert_array_equal(Y, v * np.outer(golden_c0[:, i], golden_c0[:, j]))


def test_forward_constant_blocks():
    """Rows 1..7 of C0 sum to zero: a constant block c maps to 64 c at DC only."""
    img = np.repeat(np.arange(256, dtype=np.uint8), 64).reshape(256, 8, 8).transpose(1, 0, 2).reshape(8, 2048)
    Y = orc.forward(img)
    expect = np.zeros((1, 256, 8, 8), np.int64)
    expect[0, :, 0, 0] = 64 * np.arange(256)
    np.testing.assert_array_equal(Y, expect)


def test_forward_brute_force_tiny(golden_c0):
    """16x24 random image: every block equals the printed C0 times A times C0^T."""
    img = synth.random_bytes((16, 24), seed=2)
    Y = orc.forward(img)
    for by in range(2):
        for bx in range(3):
            A = img[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].astype(np.int64)
            np.testing.assert_array_equal(Y[by, bx], golden_c0 @ A @ golden_c0.T)


def test_forward_respects_pitch():
    """A plane inside a wider buffer transforms like the cropped plane."""
    big = synth.random_bytes((16, 40), seed=4)
    np.testing.assert_array_equal(orc.forward(big[:, :16]), orc.forward(np.ascontiguousarray(big[:, :16])))


def test_shape_rejected():
    """Reading: sides that are not multiples of 8 are rejected."""
    with pytest.raises(RuntimeError):
        orc.forward(np.zeros((8, 12), np.uint8))


def test_dct_twin_matches_scipy():
    """The exact-DCT baseline: per block, scipy's orthonormal 2-D DCT."""
    img = synth.random_bytes((16, 16), seed=5)
    Y = orc.forward_f64(img, orc.KIND_DCT)
    for by in range(2):
        for bx in range(2):
            A = img[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].astype(np.float64)
            np.testing.assert_allclose(Y[by, bx], scipy.fft.dctn(A, norm="ortho"), atol=1e-10)


# ------------------------------------------------------------------ compress

def test_compress_equals_orthonormal_transform():
    """Sec. 2: S (C0 A C0^T) S = C_orth A C_orth^T; compress returns it in zigzag order."""
    img = synth.image_1f(32, 32, seed=6)
    Yc = orc.compress(orc.forward(img), 64)
    Yo = orc.forward_f64(img, orc.KIND_RDCT).reshape(-1, 64)
    np.testing.assert_allclose(Yc, Yo[:, orc.zigzag()], atol=1e-9)


def test_compress_dc_closed_form():
    """d_0^2 = 1/8, so the first retained coefficient is (block sum) / 8."""
    img = synth.random_bytes((16, 16), seed=7)
    Yc = orc.compress(orc.forward(img), 3)
    sums = img.reshape(2, 8, 2, 8).sum(axis=(1, 3)).reshape(-1)
    np.testing.assert_allclose(Yc[:, 0], sums / 8.0, rtol=1e-15)


# ------------------------------------------------------------------- inverse

@pytest.mark.parametrize("kind", [orc.KIND_RDCT, orc.KIND_DCT])
def test_exact_reconstruction_at_r64(kind):
    """Orthogonal transforms invert exactly when all 64 coefficients are kept."""
    img = synth.image_1f(64, 64, seed=8)
    xhat, u8, sse, sse_u8 = orc.fused(img, 64, kind)
    np.testing.assert_allclose(xhat, img, atol=1e-9)
    np.testing.assert_array_equal(u8, img)
    assert sse < 1e-15 and sse_u8 == 0.0


@pytest.mark.parametrize("kind", [orc.KIND_RDCT, orc.KIND_DCT])
@pytest.mark.parametrize("r", [1, 2, 5, 10, 16, 33, 45, 63])
def test_parseval(kind, r):
    """Orthogonality: the pixel-domain SSE of the reconstruction equals the energy
    of the dropped orthonormal coefficients."""
    img = synth.image_1f(32, 40, seed=9 + r)
    _, _, sse, _ = orc.fused(img, r, kind, want_xhat=False, want_u8=False)
    Y = orc.forward_f64(img, kind).reshape(-1, 64)[:, orc.zigzag()]
    dropped = np.sum(Y[:, r:] ** 2)
    assert sse == pytest.approx(dropped, rel=1e-12)


def test_inverse_matches_scipy_for_dct():
    """Exact-DCT inverse of masked coefficients equals scipy's orthonormal 2-D IDCT."""
    img = synth.image_1f(16, 16, seed=10)
    r = 10
    zz = orc.zigzag()
    Y = orc.forward_f64(img, orc.KIND_DCT).reshape(-1, 64)
    X = orc.inverse(Y[:, zz[:r]], 2, 2, r, orc.KIND_DCT)
    for b in range(4):
        by, bx = divmod(b, 2)
        Ym = np.zeros(64)
        Ym[zz[:r]] = Y[b, zz[:r]]
        ref = scipy.fft.idctn(Ym.reshape(8, 8), norm="ortho")
        np.testing.assert_allclose(X[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8], ref, atol=1e-10)


def test_inverse_of_compress_matches_fused():
    """compress -> inverse reproduces the fused reconstruction."""
    img = synth.image_1f(24, 32, seed=11)
    r = 16
    X = orc.inverse(orc.compress(orc.forward(img), r), 4, 3, r)
    xhat, _, _, _ = orc.fused(img, r)
    np.testing.assert_allclose(X, xhat, atol=1e-10)


def test_r1_rdct_equals_dct():
    """Row 0 of C_orth equals row 0 of C, so at r = 1 both give the same error."""
    img = synth.image_1f(64, 64, seed=12)
    s_r = orc.fused(img, 1, orc.KIND_RDCT, False, False)[2]
    s_d = orc.fused(img, 1, orc.KIND_DCT, False, False)[2]
    assert s_r == pytest.approx(s_d, rel=1e-13)


def test_symmetric_zone_transpose_invariance():
    """When r ends on a full anti-diagonal the retained zone is symmetric, so
    transposing the image leaves the error unchanged."""
    img = synth.image_1f(32, 32, seed=13)
    for r in FULL_DIAGONALS:
        a = orc.fused(img, r, want_xhat=False, want_u8=False)[2]
        b = orc.fused(np.ascontiguousarray(img.T), r, want_xhat=False, want_u8=False)[2]
        assert a == pytest.approx(b, rel=1e-12, abs=1e-12)


def test_u8_output_is_rounded_clamped_reconstruction():
    """Reading: the 8-bit output is clamp(rint(xhat), 0, 255)."""
    img = (synth.random_bytes((32, 32), seed=14) >= 128).astype(np.uint8) * 255  # binary noise rings
    xhat, u8, _, sse_u8 = orc.fused(img, 40)
    np.testing.assert_array_equal(u8, np.clip(np.rint(xhat), 0, 255).astype(np.uint8))
    assert sse_u8 == pytest.approx(orc.sse(img, u8))
    assert xhat.min() < 0 and xhat.max() > 255  # both clamps are exercised


def test_sse_hand_computed_on_padded_rows():
    """The squared-error sum (Sec. 3) over a plane whose rows are padded: only the w x h window counts,
    row by row.  Reference 10 everywhere and reconstruction 13 (9 per pixel) except three pixels set
    apart so that a transposed or mis-pitched walk changes the sum; the padding holds values that
    would dominate it if read."""
    h, w, pitch = 16, 24, 40
    ref_buf = np.full((h, pitch), 250, np.uint8)
    rec_buf = np.full((h, pitch), 0, np.uint8)
    ref, rec = ref_buf[:, :w], rec_buf[:, :w]
    ref[...] = 10
    rec[...] = 13
    rec[2, 5] = 20    # (20 - 10)^2 = 100
    rec[15, 23] = 0   # 100
    ref[7, 0] = 200   # (13 - 200)^2 = 34969
    expected = 9 * (h * w - 3) + 100 + 100 + 34969  # 38598
    assert orc.sse(ref, rec) == 38598 == expected
    # a float reconstruction 0.5 above: (d + 1/2)^2 = d^2 + d + 1/4, and the differences d sum to
    # 3 * 381 + 10 - 10 - 187 = 956, so the sum is 38598 + 956 + 384 / 4 = 39650
    assert orc.sse(ref, rec.astype(np.float64) + 0.5) == 39650.0


def test_sweep_matches_fused_and_is_monotone():
    """The r sweep equals the fused error at each r, decreases with r, and is 0 at 64."""
    img = synth.image_1f(16, 24, seed=15)
    s = orc.sweep(img)
    for r in (1, 7, 30, 64):
        assert s[r - 1] == pytest.approx(orc.fused(img, r, want_xhat=False, want_u8=False)[2], rel=1e-12, abs=1e-12)
    assert np.all(np.diff(s) <= 1e-9)
    assert s[63] < 1e-15


# ------------------------------------------------------------------- quality

def test_psnr_definition():
    """Sec. 3: PSNR = 10 log10(255^2 / MSE)."""
    assert orc.psnr(255.0 ** 2) == 0.0
    assert orc.psnr(255.0 ** 2 / 100.0) == pytest.approx(20.0)
    assert orc.psnr(0.0) == float("inf")
    assert orc.mse(600.0, 60) == 10.0


def test_average_and_ape():
    """Sec. 3: averages are plain means over images; APE is relative to the DCT."""
    assert orc.average([20.0, 30.0]) == 25.0
    assert orc.ape(11.0, 10.0) == pytest.approx(10.0)


def test_threads_do_not_change_results():
    img = synth.image_1f(64, 64, seed=16)
    a = orc.fused(img, 10, nthreads=1)
    b = orc.fused(img, 10, nthreads=4)
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == pytest.approx(b[2], rel=1e-12)


# ----------------------------------------------------------- UQI (Sec. 3)

def _uqi_brute(x, y, n=8):
    """UQI straight from its statistics (numpy mean / var / cov, ddof = 1), window by window."""
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    h, w = x.shape
    qs = []
    for i in range(h - n + 1):
        for j in range(w - n + 1):
            a, b = x[i:i + n, j:j + n].ravel(), y[i:i + n, j:j + n].ravel()
            c = np.cov(a, b)
            ma, mb = a.mean(), b.mean()
            d1, d2 = c[0, 0] + c[1, 1], ma * ma + mb * mb
            f1 = 1.0 if d1 == 0 else 2 * c[0, 1] / d1
            f2 = 1.0 if d2 == 0 else 2 * ma * mb / d2
            qs.append(f1 * f2)
    return float(np.mean(qs)), len(qs)


def test_uqi_identity_and_range():
    x = synth.image_1f(40, 48, seed=3)
    assert orc.uqi(x, x) == pytest.approx(1.0, abs=1e-15)
    xo, uo, _, _ = orc.fused(x, 6)
    q = orc.uqi(x, uo)
    assert -1.0 <= q < 1.0


@pytest.mark.parametrize("a", [0.5, 2.0, 3.0])
def test_uqi_scaled_copy_closed_form(a):
    # y = a x: each factor is 2a / (1 + a^2) in every window with nonzero mean and variance
    x = synth.random_bytes((24, 32), seed=4).astype(np.uint8) | 1
    q = orc.uqi(x, a * x.astype(np.float64))
    assert q == pytest.approx(4 * a * a / (1 + a * a) ** 2, rel=1e-12)


def test_uqi_shift_and_negation_closed_form():
    from scipy.ndimage import uniform_filter
    x = synth.image_1f(30, 37, seed=5).astype(np.float64)
    m = uniform_filter(x, size=8, mode="constant")  # centred 8x8 window means
    m = m[4:x.shape[0] - 3, 4:x.shape[1] - 3]        # the (h-7) x (w-7) full windows
    assert m.shape == (23, 30)
    c = 17.0
    # y = x + c: the structure factor is 1, the luminance factor depends on the window mean
    exp = np.mean(2 * m * (m + c) / (m * m + (m + c) ** 2))
    assert orc.uqi(x.astype(np.uint8), x + c) == pytest.approx(exp, rel=1e-12)
    # y = 255 - x: the structure factor is -1 wherever the window is not flat
    exp = np.mean(-2 * m * (255 - m) / (m * m + (255 - m) ** 2))
    assert orc.uqi(x.astype(np.uint8), 255.0 - x) == pytest.approx(exp, rel=1e-12)


def test_uqi_flat_windows():
    x = np.full((8, 8), 100, np.uint8)
    assert orc.uqi(x, np.full((8, 8), 100, np.uint8)) == 1.0
    # flat against flat: structure factor 1 by the zero-denominator rule, luminance 2cd/(c^2+d^2)
    assert orc.uqi(x, np.full((8, 8), 50, np.uint8)) == pytest.approx(2 * 100 * 50 / (100 ** 2 + 50 ** 2))
    z = np.zeros((9, 9), np.uint8)
    assert orc.uqi(z, z) == 1.0


@pytest.mark.parametrize("shape", [(8, 8), (9, 13), (16, 11)])
def test_uqi_brute_force_and_symmetry(shape):
    x = synth.random_bytes(shape, seed=6).astype(np.uint8)
    y = synth.random_bytes(shape, seed=7).astype(np.uint8)
    x[:, :3] = 40  # some flat-ish windows and correlated content
    y[:, :3] = 40
    y[2:, 4:] = x[2:, 4:] // 2 + 30
    q_ref, nwin = _uqi_brute(x, y)
    assert nwin == (shape[0] - 7) * (shape[1] - 7)
    assert orc.uqi(x, y) == pytest.approx(q_ref, rel=1e-12, abs=1e-14)
    assert orc.uqi(y, x) == pytest.approx(orc.uqi(x, y), rel=1e-14)


# ------------------------------------------- variants (conclusion; SDCT of Sec. 3)

def _zz_table():
    return np.array([int(v) for row in load_golden("zigzag_jpeg.txt") for v in row])


def _kron_reference(img, r, F, G):
    """Every block through vec(Y) = (F kron F) vec(A), the JPEG-order zonal mask and vec(X) = (G kron G) vec(Yhat)."""
    KF, KG = np.kron(F, F), np.kron(G, G)
    keep = np.zeros(64, bool)
    keep[_zz_table()[:r]] = True
    h, w = img.shape
    out = np.zeros((h, w))
    for by in range(h // 8):
        for bx in range(w // 8):
            a = img[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].astype(np.float64).ravel()
            y = KF @ a
            out[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8] = (KG @ np.where(keep, y, 0.0)).reshape(8, 8)
    return out


def test_variant_round_is_c_orth():
    F, G = orc.variant_matrices("round")
    np.testing.assert_allclose(F, orc.orth_matrix(), atol=1e-15)
    np.testing.assert_allclose(G, F.T, atol=0)
    img = synth.image_1f(24, 32, seed=8)
    for r in (1, 10, 45):
        xg, ug, sg, _ = orc.fused_general(img, r, F, G)
        xo, uo, so, _ = orc.fused(img, r)
        np.testing.assert_allclose(xg, xo, atol=1e-10)
        assert sg == pytest.approx(so, rel=1e-10)


@pytest.mark.parametrize("name", ["ceil", "sdct_polar"])
def test_variant_polar_factor(name):
    import scipy.linalg
    C = orc.dct_matrix()
    T = np.ceil(2 * C) if name == "ceil" else np.sign(C)
    F, G = orc.variant_matrices(name)
    np.testing.assert_allclose(F @ F.T, np.eye(8), atol=1e-13)
    np.testing.assert_array_equal(G, F.T)
    # the orthogonal factor of the polar decomposition T = P U (scipy's SVD route, not the eigen route)
    U, P = scipy.linalg.polar(T, side="left")
    np.testing.assert_allclose(F, U, atol=1e-12)
    # F T^T = P is symmetric positive definite
    Pm = F @ T.T
    np.testing.assert_allclose(Pm, Pm.T, atol=1e-12)
    assert np.linalg.eigvalsh((Pm + Pm.T) / 2).min() > 0


def test_variant_matrices_structure():
    C = orc.dct_matrix()
    # ceil(2C): first row all ones (2/sqrt(8) < 1), every other entry 0 or 1 (|2C| < 1 off the first row)
    Tc = np.ceil(2 * C)
    assert (Tc[0] == 1).all() and set(np.unique(Tc[1:])) == {0.0, 1.0}
    # floor(2C): the first row is zero, so T T^T is singular and the variant is rejected
    assert (np.floor(2 * C)[0] == 0).all()
    with pytest.raises(ValueError):
        orc.variant_matrices("floor")
    # the signed DCT: the Table 2 matrix, rebuilt by its exact inverse
    F, G = orc.variant_matrices("sdct")
    np.testing.assert_array_equal(F, orc.sdct_matrix())
    np.testing.assert_allclose(G @ F, np.eye(8), atol=1e-14)
    # its even rows are orthogonal with norm 1 after the 1/sqrt(8) scaling; its odd rows are not
    Gm = F @ F.T
    np.testing.assert_allclose(Gm[::2, ::2], np.eye(4), atol=1e-15)
    assert abs(Gm[1, 3]) == pytest.approx(0.5)


@pytest.mark.parametrize("name", ["round", "ceil", "sdct", "sdct_polar"])
def test_fused_general_against_kronecker_form(name):
    F, G = orc.variant_matrices(name)
    img = synth.random_bytes((16, 24), seed=9)
    for r in (1, 7, 30, 64):
        ref = _kron_reference(img, r, F, G)
        xg, ug, sg, su = orc.fused_general(img, r, F, G)
        np.testing.assert_allclose(xg, ref, atol=1e-9)
        assert sg == pytest.approx(float(((ref - img) ** 2).sum()), rel=1e-9, abs=1e-12)
        np.testing.assert_array_equal(ug, np.clip(np.rint(xg), 0, 255).astype(np.uint8))
    # r = 64 keeps everything: exact reconstruction (G F = I)
    assert orc.fused_general(img, 64, F, G)[2] < 1e-18 * img.size * 255 ** 2
