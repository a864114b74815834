"""The host pipeline (rdct_pipeline_run): planes in host memory, staged through device slots
(copies overlapped with kernels) or read and written in place by the kernels (direct mode:
pinned memory, and pageable memory on a device that reaches it through the host page tables).  Both must give exactly what the device-resident path gives: the same uint8
reconstruction and the same per-image error (576 * SSE is an exact integer on every route);
a few planes are also checked against the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import assert_u8_close, cuda_or_skip, pageable_direct_supported

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _planes(seed, pinned):
    """Mixed sizes, padded pitches, r per image; images 0..3 with 1-3 planes each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = [(0, 264, 1000, 16), (0, 136, 72, 16), (1, 1080, 1920, 4), (2, 8, 8, 64), (2, 520, 512, 1),
             (3, 2160, 3840, 32), (3, 1080, 1920, 32), (3, 1080, 1920, 32)]
    out = []
    for k, (img, h, w, r) in enumerate(specs):
        pitch = w + (0 if k % 2 else 40)
        a = synth.image_1f(h, w, seed=seed * 100 + k) if k != 3 else rng.integers(0, 256, (h, w), dtype=np.uint8)
        src = torch.zeros((h, pitch), dtype=torch.uint8)
        src[:, :w] = torch.from_numpy(np.ascontiguousarray(a))
        dst = torch.full((h, pitch), 7, dtype=torch.uint8)
        if pinned:
            src, dst = src.pin_memory(), dst.pin_memory()
        out.append((src[:, :w], dst[:, :w], r, img))
    return out


def _device_reference(jobs, dev):
    outs, sse = [], np.zeros(4)
    for src, _, r, img in jobs:
        u8, _, s = rdct.fused(src.contiguous().to(dev), r)
        outs.append(u8.cpu())
        sse[img] += s.item()
    return outs, sse


@pytest.mark.parametrize("mode,pinned", [(rdct.Pipeline.STAGED, False), (rdct.Pipeline.STAGED, True),
                                         (rdct.Pipeline.DIRECT, True), (rdct.Pipeline.AUTO, True),
                                         (rdct.Pipeline.AUTO, False)])
def test_pipeline_matches_device_path(dev, mode, pinned):
    jobs = _planes(1, pinned)
    ref_out, ref_sse = _device_reference(jobs, dev)
    # a small budget: 3 slots of about 2.7 MB force bands and several groups
    p = rdct.Pipeline(device_budget_bytes=8 << 20, depth=3, mode=mode)
    sse = p.run(jobs, 4)
    p.close()
    for (src, dst, r, img), ref in zip(jobs, ref_out):
        assert torch.equal(dst, ref), (src.shape, r)
    np.testing.assert_allclose(sse, ref_sse, rtol=1e-12, atol=1e-9)
    # the padding after each row is untouched
    for src, dst, r, img in jobs:
        full = dst.as_strided((dst.shape[0], dst.stride(0)), (dst.stride(0), 1))
        if full.shape[1] > dst.shape[1]:
            assert bool((full[:, dst.shape[1]:] == 7).all())


def test_pipeline_against_oracle(dev):
    jobs = _planes(2, True)
    p = rdct.Pipeline(device_budget_bytes=64 << 20, depth=2, mode=rdct.Pipeline.DIRECT)
    sse = p.run(jobs, 4)
    p.close()
    tot = np.zeros(4)
    for src, dst, r, img in jobs[:5]:
        xo, uo, so, _ = orc.fused(np.ascontiguousarray(src.numpy()), r)
        assert_u8_close(dst.numpy(), uo, xo, tie_window=1e-6)
        tot[img] += so
    for img in (0, 1, 2):
        assert sse[img] == pytest.approx(tot[img], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("mode", [rdct.Pipeline.STAGED, rdct.Pipeline.DIRECT])
def test_pipeline_u8_error(dev, mode):
    """Both modes return each image's 8-bit error: that of the planes they wrote back."""
    jobs = _planes(4, True)
    p = rdct.Pipeline(device_budget_bytes=8 << 20, depth=3, mode=mode)
    sse, sse8 = p.run(jobs, 4, want_u8_error=True)
    p.close()
    ref8 = np.zeros(4)
    for src, dst, r, img in jobs:
        ref8[img] += orc.sse(np.ascontiguousarray(src.numpy()), np.ascontiguousarray(dst.numpy()))
    np.testing.assert_array_equal(np.array(sse8), ref8)
    np.testing.assert_allclose(sse, _device_reference(jobs, dev)[1], rtol=1e-12, atol=1e-9)


def test_pipeline_sse_only_and_direct_on_pageable(dev):
    """Direct mode on pageable planes: refused where the device cannot address pageable memory, and
    otherwise exactly the device path's result."""
    jobs = [(src, None, r, img) for src, _, r, img in _planes(3, True)]
    ref = _device_reference(jobs, dev)[1]
    p = rdct.Pipeline(device_budget_bytes=32 << 20, depth=2, mode=rdct.Pipeline.DIRECT)
    np.testing.assert_allclose(p.run(jobs, 4), ref, rtol=1e-12, atol=1e-9)
    pageable = [(torch.from_numpy(src.numpy().copy()), None, r, img) for src, _, r, img in jobs]
    if pageable_direct_supported():
        np.testing.assert_allclose(p.run(pageable, 4), ref, rtol=1e-12, atol=1e-9)
    else:
        with pytest.raises(rdct.RdctError):
            p.run(pageable, 4)
    p.close()


@pytest.mark.parametrize("touched", [True, False])
def test_pipeline_direct_pageable_output(dev, touched):
    """Pageable planes in and out through the kernels (direct mode where the device supports it), with
    output buffers the host has or has not touched: the same bytes and errors as the device path."""
    if not pageable_direct_supported():
        pytest.skip("the device does not address pageable host memory")
    jobs = []
    for src, _, r, img in _planes(5, False):
        h, w = src.shape
        pitch = src.stride(0)  # one pitch for source and destination
        dst = np.full((h, pitch), 7, np.uint8) if touched else np.empty((h, pitch), np.uint8)
        jobs.append((src, torch.from_numpy(dst)[:, :w], r, img))
    ref_out, ref_sse = _device_reference(jobs, dev)
    p = rdct.Pipeline(device_budget_bytes=32 << 20, depth=2, mode=rdct.Pipeline.DIRECT)
    sse = p.run(jobs, 4)
    p.close()
    for (src, dst, r, img), ref in zip(jobs, ref_out):
        assert torch.equal(dst, ref), (src.shape, r)
    np.testing.assert_allclose(sse, ref_sse, rtol=1e-12, atol=1e-9)
