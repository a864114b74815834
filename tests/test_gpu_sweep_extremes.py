"""GPU parity of the r sweep (Sec. 3: SSE for every r), for the RDCT and for
the exact DCT, on inputs chosen for its arithmetic and its work lists.

Compared with the oracle's direct reconstructions (64 of them per plane):
random 0/255 planes (every coefficient energy near its largest), planes of
pixels near one end of the range, planes stored at an 8-byte offset and at a
pitch that is not a multiple of 16, widths that are not a multiple of 32
blocks, single block rows, and one call over many planes that share one large
buffer (a call larger than the allocation-free form accepts).  The RDCT rows
are exact (integer energies); the DCT rows meet the PSNR tolerance and, for
the same contents stored differently, agree to FP32 summation order (the DCT
pass sums each thread's blocks in FP32 and the planes' bins with atomics).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import assert_sse_close, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _rng_plane(h, w, seed, lo=0, hi=256, choices=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    if choices is not None:
        return rng.choice(np.array(choices, np.uint8), size=(h, w))
    return rng.integers(lo, hi, size=(h, w), dtype=np.uint8)


def _at_offset(img: np.ndarray, dev, offset: int, pitch: int) -> torch.Tensor:
    """The plane stored `offset` bytes into a buffer with `pitch` bytes per row."""
    h, w = img.shape
    buf = torch.full((offset + h * pitch + 64,), 91, dtype=torch.uint8, device=dev)
    view = torch.as_strided(buf, (h, w), (pitch, 1), offset)
    view.copy_(to_dev(img, dev))
    return view


KINDS = [rdct.KIND_RDCT, rdct.KIND_DCT]


def _check_against_oracle(out_row: np.ndarray, img: np.ndarray, kind=rdct.KIND_RDCT):
    ref = orc.sweep(img, kind)
    if kind == rdct.KIND_RDCT:
        np.testing.assert_allclose(out_row, ref, rtol=1e-9, atol=1e-9)
    else:
        for r in range(1, 65):
            assert_sse_close(out_row[r - 1], ref[r - 1], img.size)


def _same_contents(a: np.ndarray, b: np.ndarray, kind):
    if kind == rdct.KIND_RDCT:
        np.testing.assert_array_equal(a, b)
    else:
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("noalloc", [False, True])
def test_sweep_mixed_planes(dev, noalloc, kind):
    """Planes of every kind in one call, each against the oracle, and the same
    contents stored three ways giving equal rows (bit-identical for the RDCT)."""
    imgs = [
        _rng_plane(512, 512, 1, choices=[0, 255]),    # near-maximal energies
        _rng_plane(320, 192, 2, 253, 256),            # pixels at the top of the range
        synth.image_1f(64, 64, seed=3),
        _rng_plane(136, 72, 4),                       # width 72: a ragged strip
        _rng_plane(64, 1024, 5),
        synth.image_1f(8, 64, seed=6),                # one block row
    ]
    tens = [to_dev(i, dev) for i in imgs]
    tens.insert(2, _at_offset(imgs[0], dev, 8, 512))
    imgs.insert(2, imgs[0])
    tens.insert(4, _at_offset(imgs[1], dev, 0, 200))
    imgs.insert(4, imgs[1])
    if noalloc:
        out = torch.empty((len(tens), 64), dtype=torch.float64, device=dev)
        rdct.sweep_noalloc(tens, out, kind)
    else:
        out = rdct.sweep(tens, kind)
    o = out.cpu().numpy()
    for i, img in enumerate(imgs):
        _check_against_oracle(o[i], img, kind)
    _same_contents(o[0], o[2], kind)
    _same_contents(o[1], o[4], kind)


@pytest.mark.parametrize("kind", KINDS)
def test_sweep_many_planes_in_one_buffer(dev, kind):
    """20 descriptors of one 8192 x 8192 plane (20 M blocks in one call, more
    than the allocation-free form's 16.7 M): every row equal, and equal to the
    oracle's direct reconstruction at several r."""
    img = _rng_plane(8192, 8192, 7, choices=[0, 1, 254, 255])
    t = to_dev(img, dev)
    out = rdct.sweep([t] * 20, kind).cpu().numpy()
    for i in range(1, 20):
        _same_contents(out[i], out[0], kind)
    # a few r: 64 full reconstructions of 64 Mpixel take too long
    for r in (1, 2, 10, 33, 63, 64):
        ref = orc.fused(img, r, kind=kind, want_xhat=False, want_u8=False)[2]
        if kind == rdct.KIND_RDCT:
            assert out[0, r - 1] == pytest.approx(ref, rel=1e-9, abs=1e-9)
        else:
            assert_sse_close(out[0, r - 1], ref, img.size)


@pytest.mark.parametrize("kind", KINDS)
def test_sweep_max_plane_energy(dev, kind):
    """A 0/255 checkerboard of 8-pixel period and its complement: large energy
    at a few positions, exactly zero elsewhere; both against the oracle."""
    y, x = np.mgrid[0:256, 0:256]
    a = (((x + y) % 2) * 255).astype(np.uint8)
    b = (255 - a).astype(np.uint8)
    out = rdct.sweep([to_dev(a, dev), to_dev(b, dev)], kind).cpu().numpy()
    _check_against_oracle(out[0], a, kind)
    _check_against_oracle(out[1], b, kind)


def test_sweep_dct_tiles_across_planes(dev):
    """The DCT pass works on tiles of 128 blocks that never span two planes:
    planes of 1, 127, 128, 129 and 257 blocks (one block row each, and one
    8 x 8 plane) in one call, each against the oracle, and the same planes in
    the reverse order giving the same rows."""
    widths = [8, 127 * 8, 128 * 8, 129 * 8, 257 * 8]
    imgs = [_rng_plane(8, w, 20 + i) for i, w in enumerate(widths)]
    tens = [to_dev(i, dev) for i in imgs]
    o = rdct.sweep(tens, rdct.KIND_DCT).cpu().numpy()
    rev = rdct.sweep(tens[::-1], rdct.KIND_DCT).cpu().numpy()[::-1]
    for i, img in enumerate(imgs):
        _check_against_oracle(o[i], img, rdct.KIND_DCT)
        _same_contents(o[i], rev[i], rdct.KIND_DCT)


@pytest.mark.parametrize("kind", KINDS)
def test_sweep_many_tiny_planes(dev, kind):
    """2500 planes of 1 to 9 blocks in one call (more planes than the DCT
    pass has groups of threads, every tile partial): every row against the
    oracle."""
    rng = np.random.Generator(np.random.PCG64(11))
    shapes = [(8 * int(a), 8 * int(b)) for a, b in rng.integers(1, 4, size=(2500, 2))]
    imgs = [_rng_plane(h, w, 100 + i) for i, (h, w) in enumerate(shapes)]
    out = rdct.sweep([to_dev(i, dev) for i in imgs], kind).cpu().numpy()
    for i, img in enumerate(imgs):
        _check_against_oracle(out[i], img, kind)
