"""Parity at full size, in the launch configuration bench.py times.

The 600-frame 3840x2160 YUV 4:2:0 clip at r = 16 and the 4096-image uneven
batch are run exactly as bench.py runs them (one graph launch of a batch
plan).  The oracle then recomputes sampled 8x8 blocks one by one (uint8
output and the block's squared error), and properties that hold at any size
are checked on everything:
  * per-frame SSE of the fused path == sum over its planes of SSE(r) from the
    r sweep (an independent kernel: all 64 coefficient energies, Parseval,
    suffix sums), exactly;
  * whole sampled frames / images (every plane) match the oracle's uint8
    reconstruction and squared error.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct
from tests.gpu_helpers import assert_sse_close, assert_u8_close, cuda_or_skip

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _sample_blocks(planes, outs, frames, r, rng, n_samples):
    """Compare n_samples random 8x8 blocks against the oracle (uint8 and squared error)."""
    for _ in range(n_samples):
        f = int(rng.integers(0, frames))
        k = int(rng.integers(0, len(planes)))
        p = planes[k][f]
        h, w = p.shape
        by, bx = int(rng.integers(0, h // 8)), int(rng.integers(0, w // 8))
        blk = p[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].cpu().numpy()
        got = outs[k][f][by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].cpu().numpy()
        xo, uo, _, _ = orc.fused(np.ascontiguousarray(blk), r)
        assert_u8_close(got, uo, xo, tie_window=1e-6)


def test_video_600_frames_4k_r16(dev):
    import bench
    wl = bench.VideoWorkload(600, 16, dev)
    stream = torch.cuda.current_stream()
    wl.step(stream)
    wl.step(stream)  # graph replay, as in the timed loop
    rdct.sync(stream)
    sse = wl.sse.clone()
    # independent kernel: the sweep's SSE(16) summed over the three planes of each frame
    sw = torch.zeros(600, dtype=torch.float64, device=dev)
    for p in wl.planes:
        sw += rdct.sweep(p, rdct.KIND_RDCT)[:, 15]
    torch.cuda.synchronize()
    assert torch.allclose(sse, sw, rtol=1e-12, atol=1e-9), (sse[:4], sw[:4])
    rng = np.random.Generator(np.random.PCG64(0))
    _sample_blocks(wl.planes, wl.out, 600, 16, rng, 300)
    # whole frames against the oracle for a few frames (all planes)
    for f in (0, 299, 599):
        tot = 0.0
        for k, p in enumerate(wl.planes):
            img = p[f].cpu().numpy()
            xo, uo, so, _ = orc.fused(img, 16, want_xhat=True, want_u8=True, nthreads=0)
            assert_u8_close(wl.out[k][f].cpu().numpy(), uo, xo, tie_window=1e-6)
            tot += so
        assert sse[f].item() == pytest.approx(tot, rel=1e-9)


def test_uneven_4096_images(dev):
    from paper_1402_6034_gb300 import synth
    n = 4096
    specs = synth.uneven_specs(n, seed=0)
    pool = synth.field_u8_torch(2048, 2048, 2.0, 0, device=str(dev), planes=4)
    rng = np.random.Generator(np.random.PCG64(1))
    total = sum(sp.w * sp.h * sp.planes for sp in specs)
    src_buf = torch.empty(total, dtype=torch.uint8, device=dev)
    dst_buf = torch.empty(total, dtype=torch.uint8, device=dev)
    jobs, off = [], 0
    for i, sp in enumerate(specs):
        for p in range(sp.planes):
            k = int(rng.integers(0, 4))
            y0, x0 = int(rng.integers(0, 2048 - sp.h + 1)), int(rng.integers(0, 2048 - sp.w + 1))
            src = src_buf[off:off + sp.w * sp.h].view(sp.h, sp.w)
            src.copy_(pool[k, y0:y0 + sp.h, x0:x0 + sp.w])
            jobs.append(rdct.BatchJob(src, dst_buf[off:off + sp.w * sp.h].view(sp.h, sp.w), sp.r, i))
            off += sp.w * sp.h
    plan = rdct.BatchPlan(jobs, n)
    sse = torch.empty(n, dtype=torch.float64, device=dev)
    plan.run(sse)
    torch.cuda.synchronize()
    # independent kernel per plane: the sweep at each plane's r
    sw = torch.zeros(n, dtype=torch.float64, device=dev)
    by_r = {}
    for j in jobs:
        by_r.setdefault(j.r, []).append(j)
    for r, js in by_r.items():
        out = rdct.sweep([j.src for j in js], rdct.KIND_RDCT)[:, r - 1]
        idx = torch.tensor([j.image for j in js], device=dev)
        sw.index_add_(0, idx, out)
    torch.cuda.synchronize()
    assert torch.allclose(sse, sw, rtol=1e-12, atol=1e-9)
    # sampled whole images against the oracle
    srng = np.random.Generator(np.random.PCG64(2))
    for i in srng.choice(n, 12, replace=False):
        tot = 0.0
        for j in jobs:
            if j.image != i:
                continue
            img = j.src.cpu().numpy()
            xo, uo, so, _ = orc.fused(img, j.r)
            assert_u8_close(j.dst.cpu().numpy(), uo, xo, tie_window=1e-6)
            tot += so
        assert sse[int(i)].item() == pytest.approx(tot, rel=1e-9)


def test_plane_larger_than_2gib(dev):
    """One 65536 x 33280 plane (2.18 GB, 35.5 M blocks): byte offsets past 2^31
    in the single-plane kernel, both batch stagings (r = 16 with TMA, r = 10
    with per-thread copies), the r sweep of both transforms and the forward transform (whose
    int32 output passes 2^31 elements).  Whole-plane SSE against the oracle,
    three 16-row bands (first rows, the rows that straddle byte 2^31, last
    rows) element by element; the DCT sweep's SSE(16) against the oracle."""
    from paper_1402_6034_gb300 import synth
    h, w = 33280, 65536
    pool = synth.field_u8_torch(2048, 2048, 2.0, 7, device=str(dev), planes=4)
    rng = np.random.Generator(np.random.PCG64(3))
    img = torch.empty((h, w), dtype=torch.uint8, device=dev)
    for y in range(0, h, 2048):
        for x in range(0, w, 2048):
            k, dy, dx = (int(v) for v in rng.integers(0, [4, 2048, 2048]))
            tile = torch.roll(pool[k], shifts=(dy, dx), dims=(0, 1))
            img[y:y + 2048, x:x + 2048] = tile[:min(2048, h - y)]
    del pool
    u8, _, sse = rdct.fused(img, 16)
    d16, d10 = torch.empty_like(img), torch.empty_like(img)
    plan = rdct.BatchPlan([rdct.BatchJob(img, d16, 16, 0), rdct.BatchJob(img, d10, 10, 1)], 2)
    sse_b = torch.empty(2, dtype=torch.float64, device=dev)
    plan.run(sse_b)
    sw = rdct.sweep([img], rdct.KIND_RDCT)
    sw_d = rdct.sweep([img], rdct.KIND_DCT)  # the tensor-core pass: tiles past byte 2^31
    torch.cuda.synchronize()
    plan.close()
    assert torch.equal(u8, d16), "single-plane and batch (TMA) reconstructions differ"
    assert sse_b[0].item() == sse.item()
    assert sw[0, 15].item() == pytest.approx(sse.item(), rel=1e-12)
    assert sw[0, 9].item() == pytest.approx(sse_b[1].item(), rel=1e-12)
    del d16
    host = img.cpu().numpy()
    _, _, so16, _ = orc.fused(host, 16, want_xhat=False, want_u8=False, nthreads=0)
    _, _, so10, _ = orc.fused(host, 10, want_xhat=False, want_u8=False, nthreads=0)
    assert sse.item() == pytest.approx(so16, rel=1e-9)
    assert sse_b[1].item() == pytest.approx(so10, rel=1e-9)
    _, _, sd16, _ = orc.fused(host, 16, kind=rdct.KIND_DCT, want_xhat=False, want_u8=False, nthreads=0)
    d_np = sw_d[0].cpu().numpy()
    assert_sse_close(d_np[15], sd16, host.size)
    assert np.all(np.diff(d_np) <= 1e-6 * np.maximum(d_np[:-1], 1.0))
    Y = rdct.forward(img)
    torch.cuda.synchronize()
    assert Y.numel() > 2 ** 31
    for y0 in (0, (1 << 31) // w - 8, h - 16):
        band = np.ascontiguousarray(host[y0:y0 + 16])
        for r, got in ((16, u8), (10, d10)):
            xo, uo, _, _ = orc.fused(band, r)
            assert_u8_close(got[y0:y0 + 16].cpu().numpy(), uo, xo, tie_window=1e-6)
        assert np.array_equal(Y[y0 // 8:y0 // 8 + 2].cpu().numpy(), orc.forward(band))


def test_sweep_1024_images(dev):
    """The r sweep over 1024 images of 512 x 512 for both transforms, launched
    as bench.py launches it (one rdct_sweep_noalloc call per transform).
    Sampled images against the oracle's direct reconstruction at every r;
    on all images: SSE(r) non-increasing in r, SSE(64) = 0 for the RDCT (the
    kept set is then the whole block and the transform is orthogonal), and
    SSE(r) of the RDCT equal to the fused kernel's on a few images."""
    import bench
    imgs = bench.sweep_images(dev, 1024)
    planes = rdct.plane_array(imgs)
    out_r = torch.empty((1024, 64), dtype=torch.float64, device=dev)
    out_d = torch.empty((1024, 64), dtype=torch.float64, device=dev)
    rdct.sweep_noalloc(planes, out_r, rdct.KIND_RDCT)
    rdct.sweep_noalloc(planes, out_d, rdct.KIND_DCT)
    torch.cuda.synchronize()
    r_np, d_np = out_r.cpu().numpy(), out_d.cpu().numpy()
    for o in (r_np, d_np):
        assert np.all(np.diff(o, axis=1) <= 1e-6 * np.maximum(o[:, :-1], 1.0))
    assert np.all(r_np[:, 63] == 0.0)
    rng = np.random.Generator(np.random.PCG64(4))
    sample = [0, 63, 64, 1023] + [int(v) for v in rng.integers(0, 1024, 2)]
    for i in sample:
        img = imgs[i].cpu().numpy()
        ref_r = orc.sweep(img, rdct.KIND_RDCT, nthreads=0)
        ref_d = orc.sweep(img, rdct.KIND_DCT, nthreads=0)
        np.testing.assert_allclose(r_np[i], ref_r, rtol=1e-9, atol=1e-9)
        for r in range(1, 65):
            assert_sse_close(d_np[i, r - 1], ref_d[r - 1], img.size)
        for r in (4, 16, 45):
            assert rdct.fused(imgs[i], r, want_u8=False)[2].item() == pytest.approx(r_np[i, r - 1], rel=1e-12,
                                                                                  abs=1e-12)
