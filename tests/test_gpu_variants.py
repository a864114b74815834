"""GPU parity of the other transforms (rdct_fused_variant) against the oracle's general
block experiment Y = F A F^T, keep r, X = G Yhat G^T, with the oracle's own matrices.
Tolerances as in gpu_helpers (FP32 products on the GPU; the signed DCT's inverse has
condition number 2.4, still far inside 1e-5 of full scale)."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import PIX_ATOL, assert_sse_close, assert_u8_close, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu

NAMES = ["round", "ceil", "sdct", "sdct_polar"]


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("r", [1, 2, 6, 10, 16, 28, 45, 64])
def test_variant_against_oracle(dev, name, r):
    img = synth.image_1f(72, 136, seed=60 + r) if r % 2 else synth.random_bytes((72, 136), seed=60 + r)
    F, G = orc.variant_matrices(name)
    xo, uo, so, _ = orc.fused_general(img, r, F, G)
    u8, f32, sse = rdct.fused_variant(to_dev(img, dev), r, rdct.VARIANTS[name], want_u8=True, want_f32=True)
    assert np.abs(f32.cpu().numpy().astype(np.float64) - xo).max() <= PIX_ATOL
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-3)
    assert_sse_close(float(sse.item()), so, img.size)


@pytest.mark.parametrize("h,w", [(8, 8), (8, 264), (520, 512), (1080, 1920)])
def test_variant_shapes(dev, h, w):
    img = synth.image_1f(h, w, seed=h + w)
    F, G = orc.variant_matrices("ceil")
    xo, uo, so, _ = orc.fused_general(img, 10, F, G)
    u8, _, sse = rdct.fused_variant(to_dev(img, dev), 10, rdct.VARIANT_CEIL)
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-3)
    assert_sse_close(float(sse.item()), so, img.size)


def test_variant_round_matches_integer_path(dev):
    """C_orth through the general FP32 kernel vs the integer fused path."""
    img = synth.image_1f(512, 512, seed=4)
    t = to_dev(img, dev)
    for r in (1, 10, 16, 45):
        a = rdct.fused_variant(t, r, rdct.VARIANT_ROUND, want_u8=False)[2].item()
        b = rdct.fused(t, r, want_u8=False)[2].item()
        assert_sse_close(a, b, img.size)


def test_variant_pitched_and_sse_only(dev):
    img = synth.image_1f(64, 96, seed=5)
    buf = torch.full((64 * 101 + 64,), 7, dtype=torch.uint8, device=dev)
    v = torch.as_strided(buf, (64, 96), (101, 1))
    v.copy_(to_dev(img, dev))
    F, G = orc.variant_matrices("sdct")
    xo, uo, so, _ = orc.fused_general(img, 21, F, G)
    u8, _, sse = rdct.fused_variant(v, 21, rdct.VARIANT_SDCT)
    assert_u8_close(u8.cpu().numpy(), uo, xo, tie_window=1e-3)
    assert_sse_close(float(sse.item()), so, img.size)
    s2 = rdct.fused_variant(to_dev(img, dev), 21, rdct.VARIANT_SDCT, want_u8=False)[2].item()
    assert_sse_close(s2, so, img.size)


def test_variant_rejects(dev):
    t = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    with pytest.raises(rdct.RdctError):
        rdct.fused_variant(t, 10, rdct.VARIANT_FLOOR)
    with pytest.raises(rdct.RdctError):
        rdct.fused_variant(t, 0, rdct.VARIANT_CEIL)
    with pytest.raises(rdct.RdctError):
        rdct.fused_variant(torch.zeros((8, 12), dtype=torch.uint8, device=dev), 10, rdct.VARIANT_CEIL)
