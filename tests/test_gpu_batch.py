"""GPU parity of the batched path: uneven planes in one graph launch.

The persistent graph-captured launch must give bit-identical reconstructions
and SSE to one plain launch per plane, and both must match the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import assert_sse_close, assert_u8_close, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _batch(dev, n_images=12, seed=0, rs=(4, 10, 16, 32), lo=64, hi=264, pitch_pad=0):
    specs = synth.uneven_specs(n_images, seed=seed, lo=lo, hi=hi, rs=rs)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    pool = synth.crop_pool(pool_side=512, n=2, seed=seed)
    jobs, host = [], []
    for i, sp in enumerate(specs):
        for p in range(sp.planes):
            img = synth.crop_plane(pool, sp.h, sp.w, rng)
            pitch = sp.w + pitch_pad
            buf = torch.zeros(sp.h * pitch + 32, dtype=torch.uint8, device=dev)
            src = torch.as_strided(buf, (sp.h, sp.w), (pitch, 1))
            src.copy_(to_dev(img, dev))
            dst = torch.zeros((sp.h, sp.w), dtype=torch.uint8, device=dev)
            jobs.append(rdct.BatchJob(src, dst, sp.r, i))
            host.append((img, sp.r, i))
    return specs, jobs, host


def _check_against_oracle(specs, jobs, host, sse):
    per_image = np.zeros(len(specs))
    npix = np.zeros(len(specs))
    for j, (img, r, i) in zip(jobs, host):
        xo, uo, so, _ = orc.fused(img, r)
        if j.dst is not None:
            assert_u8_close(j.dst.cpu().numpy(), uo, xo, tie_window=1e-6)
        per_image[i] += so
        npix[i] += img.size
    for i in range(len(specs)):
        assert_sse_close(sse[i], per_image[i], int(npix[i]))
        assert sse[i] == pytest.approx(per_image[i], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("pitch_pad", [0, 8, 3])
def test_batch_graph_matches_oracle(dev, pitch_pad):
    specs, jobs, host = _batch(dev, pitch_pad=pitch_pad)
    plan = rdct.BatchPlan(jobs, len(specs))
    sse = torch.empty(len(specs), dtype=torch.float64, device=dev)
    plan.run(sse)
    plan.run(sse)  # graph replay
    rdct.sync()  # raises on an asynchronous error or a TMA wait that ran out
    _check_against_oracle(specs, jobs, host, sse.cpu().numpy())
    plan.close()


def test_batch_every_r_class(dev):
    """Plans that mix all three register classes (r up to 64)."""
    specs, jobs, host = _batch(dev, n_images=16, seed=5, rs=(1, 3, 6, 10, 15, 21, 28, 36, 45, 55, 64))
    plan = rdct.BatchPlan(jobs, len(specs))
    sse = torch.empty(len(specs), dtype=torch.float64, device=dev)
    plan.run(sse)
    torch.cuda.synchronize()
    _check_against_oracle(specs, jobs, host, sse.cpu().numpy())


def test_batch_mixed_staging(dev):
    """One plan whose planes take both stagings: from r = 16 a plane goes to
    the TMA kernel when its rows and its reconstruction start on 16-byte
    boundaries and its last 32-column segment is nearly full; the rest (r
    below 16, 8-byte pitches, a reconstruction with an 8-byte pitch, ragged
    widths) to the per-thread-copy kernel of the same r.  Each plane must match
    the oracle and the per-plane launches bit for bit."""
    shapes = [  # (h, w, src pitch, dst pitch, r)
        (64, 512, 512, 512, 16),     # TMA
        (72, 504, 504, 504, 16),     # 8-byte pitch
        (80, 480, 480, 480, 21),     # TMA, 60 of 64 segment lanes busy
        (48, 200, 208, 200, 32),     # 25 of 32 lanes busy
        (136, 1024, 1040, 1024, 45), # TMA, padded source pitch
        (40, 256, 256, 256, 10),     # r below 16
        (56, 512, 512, 520, 32),     # reconstruction with an 8-byte pitch
        (24, 2048, 2048, 2048, 64),  # TMA, odd number of block rows
        (64, 512, 512, None, 32),    # TMA, error only (no reconstruction stored)
        (64, 512, 512, None, 16),    # TMA, error only
    ]
    rng = np.random.Generator(np.random.PCG64(21))
    pool = synth.crop_pool(pool_side=512, n=2, seed=21)
    jobs, host = [], []
    for i, (h, w, sp, dp, r) in enumerate(shapes):
        img = synth.crop_plane(pool, h, w, rng)
        sbuf = torch.zeros(h * sp, dtype=torch.uint8, device=dev)
        src = torch.as_strided(sbuf, (h, w), (sp, 1))
        src.copy_(to_dev(img, dev))
        dst = None
        if dp is not None:
            dbuf = torch.zeros(h * dp, dtype=torch.uint8, device=dev)
            dst = torch.as_strided(dbuf, (h, w), (dp, 1))
        jobs.append(rdct.BatchJob(src, dst, r, i))
        host.append((img, r, i))
    specs = list(range(len(shapes)))
    # the two-block kernel (the one with both stagings), whatever the autotune cache holds
    plan = rdct.BatchPlan(jobs, len(shapes), tune={"warps_per_cta": 4, "ctas_per_sm": 0, "items_per_chunk": 16,
                                                   "blocks_per_thread": 2})
    nr = len({r for *_, r in shapes})
    assert nr + 1 <= plan.kernels_per_run() <= 2 * nr + 1  # per r: one or two stagings; + error conversion
    sse = torch.empty(len(shapes), dtype=torch.float64, device=dev)
    plan.run(sse)
    rdct.sync()
    _check_against_oracle(specs, jobs, host, sse.cpu().numpy())
    outs = [j.dst.clone() if j.dst is not None else None for j in jobs]
    sse_p = torch.empty(len(shapes), dtype=torch.float64, device=dev)
    plan.run_per_plane(sse_p)
    torch.cuda.synchronize()
    plan.close()
    assert torch.equal(sse, sse_p)
    for a, j in zip(outs, jobs):
        if a is not None:
            assert torch.equal(a, j.dst)
    # the same plan with per-thread copies for every plane (tune staging 1): no TMA launch, same results
    plan_c = rdct.BatchPlan(jobs, len(shapes), tune={"warps_per_cta": 4, "ctas_per_sm": 0, "items_per_chunk": 16,
                                                     "blocks_per_thread": 2, "staging": 1})
    assert plan_c.kernels_per_run() == nr + 1
    sse_c = torch.empty(len(shapes), dtype=torch.float64, device=dev)
    plan_c.run(sse_c)
    rdct.sync()
    plan_c.close()
    assert torch.equal(sse, sse_c)
    for a, j in zip(outs, jobs):
        if a is not None:
            assert torch.equal(a, j.dst)


def _tune(bpt):
    return {"warps_per_cta": 4 if bpt == 2 else 8, "ctas_per_sm": 0, "items_per_chunk": 16, "blocks_per_thread": bpt}


def test_dropped_coefficient_form_matches_the_scalar_kernel(dev):
    """From r = 36 the two-block kernel rebuilds each block as 576 A - C0^T (W o Y_dropped) C0 from the
    coefficients it drops; the scalar kernel still inverts the kept ones.  The two must agree bit for bit
    (reconstruction, exact SSE and the 8-bit error) at every r from 32 to 64, for planes that take TMA
    staging (16-byte aligned, full 32-column segments) and planes that take the per-thread copies (an
    8-byte pitch), each with an odd number of block rows."""
    rng = np.random.Generator(np.random.PCG64(33))
    pool = synth.crop_pool(pool_side=512, n=2, seed=33)
    jobs, host = [], []
    for k, r in enumerate(range(32, 65)):
        for (h, w, sp) in ((72, 256, 256), (40, 200, 208)):
            img = synth.crop_plane(pool, h, w, rng)
            sbuf = torch.zeros(h * sp, dtype=torch.uint8, device=dev)
            src = torch.as_strided(sbuf, (h, w), (sp, 1))
            src.copy_(to_dev(img, dev))
            dst = torch.zeros((h, w), dtype=torch.uint8, device=dev)
            jobs.append(rdct.BatchJob(src, dst, r, len(host)))
            host.append((img, r, len(host)))
    n = len(host)
    out = {}
    for bpt in (2, 1):
        plan = rdct.BatchPlan(jobs, n, tune=_tune(bpt))
        sse = torch.empty(n, dtype=torch.float64, device=dev)
        sse8 = torch.empty(n, dtype=torch.float64, device=dev)
        plan.run(sse, sse_u8=sse8)
        rdct.sync()
        out[bpt] = (sse.clone(), sse8.clone(), [j.dst.clone() for j in jobs])
        plan.close()
    assert torch.equal(out[2][0], out[1][0])
    assert torch.equal(out[2][1], out[1][1])
    for a, b in zip(out[2][2], out[1][2]):
        assert torch.equal(a, b)
    _check_against_oracle(list(range(n)), jobs, host, out[2][0].cpu().numpy())
    for (img, r, i), d in zip(host, out[2][2]):
        assert out[2][1][i].item() == orc.sse(img, d.cpu().numpy())


def test_batch_u8_error_every_staging(dev):
    """The 8-bit error per image from the graph launch equals that of the returned planes (summed over
    an image's planes), for both stagings and both forms, and asking for it changes nothing else."""
    specs, jobs, host = _batch(dev, n_images=14, seed=17, rs=(4, 16, 21, 32, 40, 57, 64), lo=64, hi=520)
    n = len(specs)
    plan = rdct.BatchPlan(jobs, n)
    sse = torch.empty(n, dtype=torch.float64, device=dev)
    sse8 = torch.empty(n, dtype=torch.float64, device=dev)
    plan.run(sse, sse_u8=sse8)
    rdct.sync()
    outs = [j.dst.clone() for j in jobs]
    ref8 = np.zeros(n)
    for (img, r, i), d in zip(host, outs):
        ref8[i] += orc.sse(img, d.cpu().numpy())
    np.testing.assert_array_equal(sse8.cpu().numpy(), ref8)
    sse_plain = torch.empty(n, dtype=torch.float64, device=dev)
    plan.run(sse_plain)  # a second graph without the 8-bit error
    sse_pp = torch.empty(n, dtype=torch.float64, device=dev)
    sse8_pp = torch.empty(n, dtype=torch.float64, device=dev)
    plan.run_per_plane(sse_pp, sse_u8=sse8_pp)
    torch.cuda.synchronize()
    plan.close()
    assert torch.equal(sse, sse_plain) and torch.equal(sse, sse_pp) and torch.equal(sse8, sse8_pp)
    for a, j in zip(outs, jobs):
        assert torch.equal(a, j.dst)


def test_batch_equals_per_plane(dev):
    specs, jobs, host = _batch(dev, n_images=20, seed=9)
    plan = rdct.BatchPlan(jobs, len(specs), tune={"warps_per_cta": 4, "ctas_per_sm": 2, "items_per_chunk": 3})
    sse_b = torch.empty(len(specs), dtype=torch.float64, device=dev)
    plan.run(sse_b)
    outs_b = [j.dst.clone() for j in jobs]
    for j in jobs:
        j.dst.zero_()
    sse_p = torch.empty(len(specs), dtype=torch.float64, device=dev)
    plan.run_per_plane(sse_p)
    torch.cuda.synchronize()
    assert torch.equal(sse_b, sse_p)
    for a, j in zip(outs_b, jobs):
        assert torch.equal(a, j.dst)


def test_autotune_picks_a_valid_shape(dev, tmp_path):
    specs, jobs, host = _batch(dev, n_images=8, seed=11)
    t = rdct.autotune(jobs, len(specs))
    assert 1 <= t["warps_per_cta"] <= 32 and t["items_per_chunk"] >= 1 and t["staging"] in (0, 1)
    plan = rdct.BatchPlan(jobs, len(specs))  # picks the cached tune
    assert plan.tune == t
    # the cache survives a save, a clear and a load (as another process would see it)
    path = str(tmp_path / "tune_cache.jsonl")
    rdct.autotune_cache_save(path)
    rdct.autotune_cache_clear()
    assert rdct.autotune_cache_load(path) >= 1
    assert rdct.BatchPlan(jobs, len(specs)).tune == t
    sse = torch.empty(len(specs), dtype=torch.float64, device=dev)
    plan.run(sse)
    torch.cuda.synchronize()
    _check_against_oracle(specs, jobs, host, sse.cpu().numpy())


def test_batch_rejects_bad_jobs(dev):
    src = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    with pytest.raises(rdct.RdctError):
        rdct.BatchPlan([rdct.BatchJob(src, None, 0, 0)], 1)
    with pytest.raises(rdct.RdctError):
        rdct.BatchPlan([rdct.BatchJob(src, None, 10, 3)], 1)
