"""GPU tests of the continuous-batching server.

Results must match the oracle, and each request's result must be identical
whether it ran alone or mixed into batches with others.  Admission must hold
the device budget, refuse what can never fit, survive injected allocation
failures (made on the host, no GPU fault), and support cancel / timeout.
"""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import assert_sse_close, assert_u8_close, cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _requests(n, seed, lo=64, hi=512):
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = synth.crop_pool(pool_side=512, n=2, seed=seed)
    reqs = []
    for i in range(n):
        side_h = int(8 * rng.integers(lo // 8, hi // 8 + 1))
        side_w = int(8 * rng.integers(lo // 8, hi // 8 + 1))
        planes = int(rng.choice([1, 3]))
        r = int(rng.integers(1, 65))
        src = np.stack([synth.crop_plane(pool, side_h, side_w, rng) for _ in range(planes)])
        reqs.append((torch.from_numpy(src).pin_memory(), r))
    return reqs


def _oracle(src, r):
    sse, outs = 0.0, []
    for p in range(src.shape[0]):
        xo, uo, so, _ = orc.fused(src[p].numpy(), r)
        sse += so
        outs.append((xo, uo))
    return sse, outs


def _run(server, reqs):
    outs = [torch.zeros_like(s).pin_memory() for s, _ in reqs]
    tickets = [server.submit(s, r, o) for (s, r), o in zip(reqs, outs)]
    res = [server.wait(t) for t in tickets]
    return outs, res


def test_results_match_oracle(dev):
    reqs = _requests(12, seed=1)
    srv = rdct.Server(device_budget_bytes=256 << 20, max_batch=8, streams=2)
    outs, res = _run(srv, reqs)
    for (src, r), out, rr in zip(reqs, outs, res):
        sse, per_plane = _oracle(src, r)
        assert_sse_close(rr["sse"], sse, src.numel())
        assert rr["sse"] == pytest.approx(sse, rel=1e-9, abs=1e-9)
        for p, (xo, uo) in enumerate(per_plane):
            assert_u8_close(out[p].numpy(), uo, xo, tie_window=1e-6)
        # the 8-bit error is that of the image returned
        assert rr["sse_u8"] == sum(orc.sse(src[p].numpy(), out[p].numpy()) for p in range(src.shape[0]))
        assert rr["mse_u8"] == pytest.approx(rr["sse_u8"] / src.numel(), rel=1e-15)
    st = srv.stats()
    assert st["completed"] == 12 and st["p999_us"] >= st["p99_us"] >= st["p50_us"] > 0
    srv.close()


def test_pageable_requests_equal_pinned(dev):
    """Requests whose planes live in plain pageable memory (moved by copy kernels where the device reaches
    such memory through the host page tables, else by the driver's copies), with padded pitches and a
    plane stride: results and images identical to the same requests in pinned memory."""
    reqs = _requests(8, seed=5)
    srv = rdct.Server(device_budget_bytes=256 << 20, max_batch=4, streams=2)
    ref_outs, ref_res = _run(srv, reqs)
    pageable, outs, tickets = [], [], []
    for src, r in reqs:
        p, h, w = src.shape
        buf = np.full((p, h + 2, w + 40), 5, np.uint8)  # padded rows and a gap between planes
        buf[:, :h, :w] = src.numpy()
        view = torch.from_numpy(buf)[:, :h, :w]
        out_buf = torch.from_numpy(np.full((p, h + 2, w + 40), 9, np.uint8))
        pageable.append((view, r))
        outs.append(out_buf)
        tickets.append(srv.submit(view, r, out_buf[:, :h, :w]))
    res = [srv.wait(t) for t in tickets]
    for (view, r), out_buf, ref_out, rr, ref in zip(pageable, outs, ref_outs, res, ref_res):
        p, h, w = view.shape
        assert torch.equal(out_buf[:, :h, :w], ref_out)
        assert bool((out_buf[:, h:, :] == 9).all()) and bool((out_buf[:, :, w:] == 9).all())
        assert rr["sse"] == ref["sse"] and rr["sse_u8"] == ref["sse_u8"]
    srv.close()


def test_alone_equals_mixed(dev):
    reqs = _requests(16, seed=2)
    alone = []
    for s, r in reqs:
        srv = rdct.Server(device_budget_bytes=64 << 20, max_batch=1, streams=1)
        alone.append(_run(srv, [(s, r)]))
        srv.close()
    srv = rdct.Server(device_budget_bytes=64 << 20, max_batch=16, streams=3)
    outs, res = _run(srv, reqs)
    assert srv.stats()["batches"] < len(reqs)  # they really were batched
    srv.close()
    for (o_a, r_a), o_m, r_m in zip(alone, outs, res):
        assert r_a[0]["sse"] == r_m["sse"] and r_a[0]["sse_u8"] == r_m["sse_u8"]
        assert torch.equal(o_a[0], o_m)


def test_admission_under_tiny_budget(dev):
    reqs = _requests(10, seed=3, lo=256, hi=512)
    need = max(2 * s.numel() for s, _ in reqs)
    budget = max(need + 4096, 1 << 20)
    srv = rdct.Server(device_budget_bytes=budget, max_batch=8, streams=2)
    outs, res = _run(srv, reqs)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["peak_resident_bytes"] <= budget
    too_big = torch.zeros((3, 1024, 1024), dtype=torch.uint8)
    with pytest.raises(rdct.RdctError) as e:
        srv.submit(too_big, 10)
    assert e.value.status == 4
    srv.close()
    for (src, r), out, rr in zip(reqs, outs, res):
        sse, _ = _oracle(src, r)
        assert rr["sse"] == pytest.approx(sse, rel=1e-9)


def test_queue_full_is_busy(dev):
    src = torch.zeros((1, 64, 64), dtype=torch.uint8).pin_memory()
    srv = rdct.Server(device_budget_bytes=1 << 20, max_batch=1, queue_capacity=2, streams=1)
    srv.inject_alloc_failures(1 << 30)  # hold everything in the queue
    t1, t2 = srv.submit(src, 5), srv.submit(src, 5)
    with pytest.raises(rdct.RdctError) as e:
        srv.submit(src, 5)
    assert e.value.status == 7
    srv.inject_alloc_failures(0)
    srv.wait(t1)
    srv.wait(t2)
    srv.close()


def test_injected_alloc_failures_keep_requests_queued(dev):
    reqs = _requests(6, seed=4)
    srv = rdct.Server(device_budget_bytes=256 << 20, max_batch=4, streams=2)
    srv.inject_alloc_failures(5)
    outs, res = _run(srv, reqs)
    assert srv.stats()["completed"] == 6
    for (src, r), rr in zip(reqs, res):
        assert rr["sse"] == pytest.approx(_oracle(src, r)[0], rel=1e-9)
    srv.close()


def test_cancel_and_timeout(dev):
    src = torch.zeros((1, 64, 64), dtype=torch.uint8).pin_memory()
    srv = rdct.Server(device_budget_bytes=1 << 20, max_batch=1, streams=1)
    srv.inject_alloc_failures(1 << 30)
    t = srv.submit(src, 7)
    with pytest.raises(rdct.RdctError) as e:
        srv.wait(t, timeout_us=1000)
    assert e.value.status == 6  # still pending
    srv.cancel(t)
    with pytest.raises(rdct.RdctError) as e:
        srv.wait(t)
    assert e.value.status == 9
    with pytest.raises(rdct.RdctError) as e:
        srv.wait(t)  # retired
    assert e.value.status == 8
    srv.inject_alloc_failures(0)
    t2 = srv.submit(src, 7)
    assert srv.wait(t2)["sse"] == 0.0  # a constant image keeps all its energy at r >= 1
    srv.close()


def test_concurrent_submitters(dev):
    import threading
    reqs = _requests(24, seed=5, lo=64, hi=256)
    srv = rdct.Server(device_budget_bytes=64 << 20, max_batch=8, streams=2)
    outs = [torch.zeros_like(s).pin_memory() for s, _ in reqs]
    results = [None] * len(reqs)

    def worker(k):
        for i in range(k, len(reqs), 4):
            s, r = reqs[i]
            results[i] = srv.wait(srv.submit(s, r, outs[i]))

    ths = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    srv.close()
    for (src, r), rr in zip(reqs, results):
        assert rr["sse"] == pytest.approx(_oracle(src, r)[0], rel=1e-9)
