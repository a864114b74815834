"""GPU parity: every C-ABI step of the path against the FP64 oracle.

Sizes span several warp strips and ragged tails (widths that are not a
multiple of 32 blocks), padded and odd pitches, and the degenerate cases
(one block, r = 1, r = 64).  Tolerances are documented in gpu_helpers.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import (PIX_ATOL, assert_coef_close, assert_sse_close, assert_u8_close, block_norms,
                               cuda_or_skip, to_dev)

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8), (16, 24), (72, 136), (128, 512), (512, 512)]


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _img(h, w, seed, kind="1f"):
    return synth.image_1f(h, w, seed=seed) if kind == "1f" else synth.random_bytes((h, w), seed=seed)


def _padded(img: np.ndarray, dev, pitch: int) -> torch.Tensor:
    """The plane stored with `pitch` bytes per row; returns the [h, w] view."""
    h, w = img.shape
    buf = torch.full((h * pitch + 64,), 77, dtype=torch.uint8, device=dev)
    view = torch.as_strided(buf, (h, w), (pitch, 1))
    view.copy_(to_dev(img, dev))
    return view


# ------------------------------------------------------------------ forward

@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("kind", ["1f", "noise"])
def test_forward_bit_exact(dev, h, w, kind):
    img = _img(h, w, 100 + h + w, kind)
    Y = rdct.forward(to_dev(img, dev)).cpu().numpy()
    np.testing.assert_array_equal(Y, orc.forward(img))


@pytest.mark.parametrize("pitch_extra", [1, 8, 16, 13])
def test_forward_pitches(dev, pitch_extra):
    img = _img(40, 264, 7, "noise")
    t = _padded(img, dev, 264 + pitch_extra)
    np.testing.assert_array_equal(rdct.forward(t).cpu().numpy(), orc.forward(img))


def test_forward_extremes(dev):
    """All-255 and all-0 blocks and an impulse: the largest |Y| = 16320."""
    img = np.zeros((16, 16), np.uint8)
    img[:8, :8] = 255
    img[8, 8] = 255
    Y = rdct.forward(to_dev(img, dev)).cpu().numpy()
    np.testing.assert_array_equal(Y, orc.forward(img))
    assert Y[0, 0, 0, 0] == 16320


@pytest.mark.parametrize("kind", [rdct.KIND_RDCT, rdct.KIND_DCT])
@pytest.mark.parametrize("h,w", [(16, 24), (72, 136), (512, 512)])
def test_forward_f32(dev, kind, h, w):
    img = _img(h, w, 3 + h, "noise")
    Yg = rdct.forward_f32(to_dev(img, dev), kind).cpu().numpy().reshape(-1, 64)
    Yo = orc.forward_f64(img, kind).reshape(-1, 64)
    assert_coef_close(Yg.astype(np.float64), Yo, block_norms(img))


# ----------------------------------------------------------------- compress

@pytest.mark.parametrize("r", [1, 2, 10, 16, 45, 64])
def test_compress(dev, r):
    img = _img(72, 136, 11 + r)
    Y = orc.forward(img)
    Yc = rdct.compress(to_dev(Y, dev), r).cpu().numpy().astype(np.float64)
    ref = orc.compress(Y, r)
    nrm = block_norms(img)
    assert_coef_close(np.pad(Yc, ((0, 0), (0, 64 - r))), np.pad(ref, ((0, 0), (0, 64 - r))), nrm)


# ------------------------------------------------------------------ inverse

@pytest.mark.parametrize("kind", [rdct.KIND_RDCT, rdct.KIND_DCT])
@pytest.mark.parametrize("r", [1, 5, 10, 16, 33, 64])
def test_inverse(dev, kind, r):
    img = _img(72, 136, 21 + r)
    nbw, nbh = 136 // 8, 72 // 8
    zz = orc.zigzag()
    if kind == rdct.KIND_RDCT:
        Yc = orc.compress(orc.forward(img), r)
    else:
        Yc = orc.forward_f64(img, kind).reshape(-1, 64)[:, zz[:r]]
    xo = orc.inverse(Yc, nbw, nbh, r, kind)
    u8, f32 = rdct.inverse(to_dev(Yc.astype(np.float32), dev), nbw, nbh, r, kind, want_u8=True, want_f32=True)
    f32 = f32.cpu().numpy().astype(np.float64)
    assert np.abs(f32 - xo).max() <= PIX_ATOL
    uo = np.clip(np.rint(xo), 0, 255).astype(np.uint8)
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-3)


# -------------------------------------------------------------------- fused

@pytest.mark.parametrize("r", list(range(1, 65)))
def test_fused_every_r(dev, r):
    """Every r (all 15 anti-diagonal classes, every partial diagonal)."""
    img = _img(72, 136, 1000 + r, "noise" if r % 2 else "1f")
    xo, uo, so, _ = orc.fused(img, r)
    u8, f32, sse = rdct.fused(to_dev(img, dev), r, want_u8=True, want_f32=True)
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-6)
    assert np.abs(f32.cpu().numpy().astype(np.float64) - xo).max() <= PIX_ATOL
    assert_sse_close(float(sse.item()), so, img.size)
    # integer route: 576 * SSE is exact, so agreement is far tighter than 1e-3 dB
    assert float(sse.item()) == pytest.approx(so, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("r", list(range(1, 65)))
def test_fused_two_block_kernel_every_r_with_u8_error(dev, r):
    """The two-block kernel (uint8 output, no FP32 output) at every r: the reconstruction from the
    kept coefficients up to r = 32 and from the dropped ones above, and the squared error of the
    8-bit reconstruction.  9 block rows, so the last row pair has one block."""
    img = _img(72, 136, 2000 + r, "noise" if r % 2 else "1f")
    xo, uo, so, s8o = orc.fused(img, r)
    t = to_dev(img, dev)
    sse8 = torch.empty(1, dtype=torch.float64, device=dev)
    u8, _, sse = rdct.fused(t, r, sse_u8=sse8)
    g = u8.cpu().numpy()
    assert_u8_close(g, uo, xo, tie_window=1e-6)
    assert float(sse.item()) == pytest.approx(so, rel=1e-9, abs=1e-9)
    # exactly the error of the 8-bit image returned, and the oracle's wherever no pixel sits at a half
    assert float(sse8.item()) == orc.sse(img, g)
    if np.array_equal(g, uo):
        assert float(sse8.item()) == s8o
    # error only: nothing stored, the same two errors
    sse8b = torch.empty(1, dtype=torch.float64, device=dev)
    _, _, sseb = rdct.fused(t, r, want_u8=False, sse_u8=sse8b)
    assert float(sseb.item()) == float(sse.item()) and float(sse8b.item()) == float(sse8.item())
    # without the 8-bit error the reconstruction and the error are the same
    u8c, _, ssec = rdct.fused(t, r)
    assert torch.equal(u8c, u8) and float(ssec.item()) == float(sse.item())


@pytest.mark.parametrize("kind", [rdct.KIND_RDCT, rdct.KIND_DCT])
@pytest.mark.parametrize("r", [1, 10, 33, 64])
def test_u8_error_with_fp32_output(dev, kind, r):
    """The single-block kernels (FP32 output, exact DCT) report the 8-bit error too."""
    img = _img(40, 264, 300 + r)
    sse8 = torch.empty(1, dtype=torch.float64, device=dev)
    u8, f32, _ = rdct.fused(to_dev(img, dev), r, kind, want_u8=True, want_f32=True, sse_u8=sse8)
    assert float(sse8.item()) == orc.sse(img, u8.cpu().numpy())
    sse8b = torch.empty(1, dtype=torch.float64, device=dev)
    rdct.fused(to_dev(img, dev), r, kind, want_u8=False, want_f32=True, sse_u8=sse8b)
    assert float(sse8b.item()) == float(sse8.item())


@pytest.mark.parametrize("h,w", SHAPES + [(2048, 2048)])
@pytest.mark.parametrize("r", [1, 10, 16, 64])
def test_fused_shapes(dev, h, w, r):
    img = _img(h, w, 7 * h + w + r)
    xo, uo, so, _ = orc.fused(img, r)
    u8, _, sse = rdct.fused(to_dev(img, dev), r)
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-6)
    assert_sse_close(float(sse.item()), so, img.size)


def test_fused_config_512_r10(dev):
    """The 512 x 512, r = 10 single-image case: PSNR within 1e-3 dB, uint8 within 1 LSB."""
    img = synth.image_1f(512, 512, alpha=2.0, seed=0)
    xo, uo, so, _ = orc.fused(img, 10)
    u8, _, sse = rdct.fused(to_dev(img, dev), 10)
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-6)
    assert_sse_close(float(sse.item()), so, img.size)


@pytest.mark.parametrize("pitch", [137, 144, 160])
def test_fused_pitched_and_unaligned(dev, pitch):
    img = _img(40, 136, pitch)
    t = _padded(img, dev, pitch)
    xo, uo, so, _ = orc.fused(img, 16)
    dst = torch.as_strided(torch.zeros(40 * pitch + 64, dtype=torch.uint8, device=dev), (40, 136), (pitch, 1))
    _, _, sse = rdct.fused(t, 16, out_u8=dst)
    assert_u8_close(dst.cpu().numpy(), uo, xo, tie_window=1e-6)
    assert float(sse.item()) == pytest.approx(so, rel=1e-9)


def test_fused_sse_only_and_r64(dev):
    img = _img(64, 64, 5, "noise")
    _, _, sse = rdct.fused(to_dev(img, dev), 64, want_u8=False)
    assert float(sse.item()) == 0.0
    u8, _, sse = rdct.fused(to_dev(img, dev), 64)
    np.testing.assert_array_equal(u8.cpu().numpy(), img)


@pytest.mark.parametrize("r", [1, 3, 10, 16, 40, 64])
def test_fused_dct(dev, r):
    img = _img(72, 136, 50 + r)
    xo, uo, so, _ = orc.fused(img, r, orc.KIND_DCT)
    u8, f32, sse = rdct.fused(to_dev(img, dev), r, rdct.KIND_DCT, want_u8=True, want_f32=True)
    assert np.abs(f32.cpu().numpy().astype(np.float64) - xo).max() <= PIX_ATOL
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-3)
    assert_sse_close(float(sse.item()), so, img.size)


def test_r1_rdct_equals_dct_on_gpu(dev):
    img = _img(64, 64, 9)
    a = rdct.fused(to_dev(img, dev), 1, rdct.KIND_RDCT, want_u8=False)[2].item()
    b = rdct.fused(to_dev(img, dev), 1, rdct.KIND_DCT, want_u8=False)[2].item()
    assert a == pytest.approx(b, rel=1e-5)


# --------------------------------------------------------------- mse / psnr

def test_mse_psnr(dev):
    img = _img(72, 136, 31)
    xo, uo, _, _ = orc.fused(img, 10)
    mse, ps = rdct.mse_psnr(to_dev(img, dev), to_dev(uo, dev))
    ref = orc.sse(img, uo) / img.size
    assert mse.item() == pytest.approx(ref, rel=1e-12)
    assert ps.item() == pytest.approx(orc.psnr(ref), abs=1e-9)
    mse_f, _ = rdct.mse_psnr(to_dev(img, dev), to_dev(xo.astype(np.float32), dev))
    assert_sse_close(mse_f.item() * img.size, orc.sse(img, xo), img.size)
    m0, p0 = rdct.mse_psnr(to_dev(img, dev), to_dev(img, dev))
    assert m0.item() == 0.0 and p0.item() == float("inf")


# ---------------------------------------------------------------------- UQI

@pytest.mark.parametrize("h,w", [(8, 8), (72, 136), (512, 512), (264, 1000)])
@pytest.mark.parametrize("r", [1, 6, 16])
def test_uqi(dev, h, w, r):
    img = _img(h, w, 90 + r)
    xo, uo, _, _ = orc.fused(img, r)
    t = to_dev(img, dev)
    # uint8 reconstruction: exact integer window sums, only the mean's summation order differs
    q = rdct.uqi(t, to_dev(uo, dev)).item()
    assert q == pytest.approx(orc.uqi(img, uo), rel=1e-12, abs=1e-14)
    # float reconstruction: the same float32 values on both sides, double window sums
    xf = xo.astype(np.float32)
    qf = rdct.uqi(t, to_dev(xf, dev)).item()
    assert qf == pytest.approx(orc.uqi(img, xf.astype(np.float64)), rel=1e-9, abs=1e-12)


def test_uqi_pitched_identity_and_flat(dev):
    img = _img(72, 136, 95)
    v = _padded(img, dev, 160)
    assert rdct.uqi(v, v).item() == pytest.approx(1.0, abs=1e-15)
    rec = _padded(orc.fused(img, 3)[1], dev, 144)
    assert rdct.uqi(v, rec).item() == pytest.approx(orc.uqi(img, orc.fused(img, 3)[1]), rel=1e-12)
    flat = torch.full((16, 16), 100, dtype=torch.uint8, device=dev)
    half = torch.full((16, 16), 50, dtype=torch.uint8, device=dev)
    assert rdct.uqi(flat, half).item() == pytest.approx(2 * 100 * 50 / (100 ** 2 + 50 ** 2), rel=1e-15)


# -------------------------------------------------------------------- sweep

@pytest.mark.parametrize("kind", [rdct.KIND_RDCT, rdct.KIND_DCT])
def test_sweep(dev, kind):
    imgs = [_img(64, 64, 70 + i) for i in range(3)] + [_img(72, 136, 80)]
    out = rdct.sweep([to_dev(i, dev) for i in imgs], kind).cpu().numpy()
    for i, img in enumerate(imgs):
        ref = orc.sweep(img, kind)
        for r in range(1, 65):
            assert_sse_close(out[i, r - 1], ref[r - 1], img.size)
        if kind == rdct.KIND_RDCT:
            np.testing.assert_allclose(out[i], ref, rtol=1e-9, atol=1e-9)


def test_sweep_matches_fused_on_gpu(dev):
    """Energy shortcut (Parseval) vs direct reconstruction, both on the GPU."""
    img = synth.image_1f(512, 512, seed=3)
    t = to_dev(img, dev)
    s = rdct.sweep([t], rdct.KIND_RDCT).cpu().numpy()[0]
    for r in (1, 10, 16, 45, 64):
        assert rdct.fused(t, r, want_u8=False)[2].item() == pytest.approx(s[r - 1], rel=1e-12, abs=1e-12)


# -------------------------------------------------------------------- errors

def test_rejects_bad_shapes_and_args(dev):
    with pytest.raises(rdct.RdctError) as e:
        rdct.fused(torch.zeros((8, 12), dtype=torch.uint8, device=dev), 10)
    assert e.value.status == 2
    with pytest.raises(rdct.RdctError) as e:
        rdct.fused(torch.zeros((8, 8), dtype=torch.uint8, device=dev), 0)
    assert e.value.status == 1
    with pytest.raises(rdct.RdctError):
        rdct.fused(torch.zeros((8, 8), dtype=torch.uint8, device=dev), 65)
