"""rdct_sweep_noalloc, the r sweep for callers that cannot allocate device memory.

Some callers cannot let a library allocate device memory when they call it:
a framework that owns the device heap through its own allocator, a real-time
loop where an allocation could stall or synchronise the device, a plug-in
whose host process forbids device allocation.  rdct_sweep_noalloc keeps its
tables in a fixed device array inside the library instead.  This file checks,
through the C-ABI, that two calls in a row give the same results as
rdct_sweep (the second call with different planes, so stale tables from the
first would show), that oversized calls are refused, and that a call really
takes no memory from the device's stream-ordered pool (where rdct_sweep takes
its tables) and leaves the free device memory unchanged.

It sits in its own file, collected last, and passes both alone in a fresh
process and after the other tests.
"""
import ctypes
import glob
import os

import numpy as np
import pytest
import torch

from paper_1402_6034_gb300 import rdct, synth
from tests.gpu_helpers import assert_sse_close, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = cuda_or_skip()
    rdct.load()
    return d


def _planes(dev, shapes, seed):
    return [to_dev(synth.image_1f(h, w, seed=seed + i), dev) for i, (h, w) in enumerate(shapes)]


@pytest.mark.parametrize("kind", [rdct.KIND_RDCT, rdct.KIND_DCT])
def test_noalloc_matches_sweep_on_two_calls(dev, kind):
    first = _planes(dev, [(512, 512), (72, 136), (64, 64), (256, 1024)], seed=40)
    second = _planes(dev, [(136, 72), (8, 8)], seed=90)
    for planes in (first, second):
        out = torch.full((len(planes), 64), -1.0, dtype=torch.float64, device=dev)
        rdct.sweep_noalloc(planes, out, kind)
        ref = rdct.sweep(planes, kind)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        for i, p in enumerate(planes):
            for r in range(1, 65):
                assert_sse_close(got[i, r - 1], want[i, r - 1], p.numel())
        if kind == rdct.KIND_RDCT:  # integer energies: exact on both paths
            np.testing.assert_array_equal(got, want)


def test_noalloc_rejects_oversized_calls(dev):
    small = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    out = torch.zeros((2049, 64), dtype=torch.float64, device=dev)
    with pytest.raises(rdct.RdctError) as e:
        rdct.sweep_noalloc([small] * 2049, out)
    assert e.value.status == 4
    # 2048 planes of 272 block rows x 32 blocks need 17 chunks each: 34816 > 32768
    tall = torch.zeros((8 * 16 * 17, 8 * 32), dtype=torch.uint8, device=dev)
    out2 = torch.zeros((2048, 64), dtype=torch.float64, device=dev)
    with pytest.raises(rdct.RdctError) as e:
        rdct.sweep_noalloc([tall] * 2048, out2)
    assert e.value.status == 4


def _cudart():
    """The CUDA runtime as a shared library (for the memory-pool counters; the library under test
    links its own copy, and both see the same device pool)."""
    cands = []
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d:
            cands += sorted(glob.glob(os.path.join(d, "lib64", "libcudart.so*")))
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.skip("libcudart not found")


class _PoolHigh:
    """Use of the current device's default memory pool: its high-water mark (cudaMemPoolAttrUsedMemHigh)
    and the memory in use now (cudaMemPoolAttrUsedMemCurrent; earlier work may still hold some)."""

    USED_MEM_CURRENT = 7
    USED_MEM_HIGH = 8

    def __init__(self):
        self.rt = _cudart()
        dev = ctypes.c_int()
        assert self.rt.cudaGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def reset(self):
        zero = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def _get(self, attr) -> int:
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def high(self) -> int:
        return self._get(self.USED_MEM_HIGH)

    def current(self) -> int:
        return self._get(self.USED_MEM_CURRENT)


def test_noalloc_takes_no_device_memory(dev):
    planes = _planes(dev, [(512, 512), (256, 1024)], seed=70)
    arr = rdct.plane_array(planes)
    out = torch.zeros((len(planes), 64), dtype=torch.float64, device=dev)
    rdct.sweep_noalloc(arr, out)  # warm: the first call on a device looks up the array's address
    torch.cuda.synchronize()
    pool = _PoolHigh()
    # control: rdct_sweep takes its tables from the stream-ordered pool (the mark is reset to the
    # memory in use now, which earlier work in the process may still hold)
    pool.reset()
    base = pool.current()
    rdct.sweep(planes)
    torch.cuda.synchronize()
    assert pool.high() > base
    # the allocation-free call takes nothing from it, and the free device memory does not move
    pool.reset()
    base = pool.current()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rdct.sweep_noalloc(arr, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert pool.high() == base
    assert free1 == free0
