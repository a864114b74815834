"""Helpers shared by the GPU parity tests: tolerances and comparisons.

Tolerances (derivations):
  * int32 coefficients: bit-exact (integer additions on both sides).
  * FP32 orthonormal coefficients: |gpu - oracle| <= 1e-5 * max(|oracle|, ||block||_2 / 8).
    The GPU forms each value with at most ~20 FP32 roundings of terms bounded by
    the block norm; the floor ||block||/8 avoids an ill-posed relative test on
    coefficients that are zero up to rounding.
  * FP32 reconstructions: |gpu - oracle| <= 1e-5 * 255 per pixel (1e-5 of full scale).
  * uint8 reconstructions: <= 1 LSB everywhere, and equal wherever the oracle's
    unrounded value is not within FP32 reach of a half (exact halves may round
    either way on either side).
  * SSE / PSNR: |dPSNR| <= 1e-3 dB; where the oracle MSE < 1e-10 (r = 64), the
    GPU MSE must be <= 1e-6 (exactly 0 on the integer path).
"""
import numpy as np
import pytest
import torch

PSNR_TOL_DB = 1e-3
COEF_RTOL = 1e-5
PIX_ATOL = 1e-5 * 255.0


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a: np.ndarray, dev) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def psnr(mse: float) -> float:
    return float("inf") if mse == 0 else 10.0 * np.log10(255.0 ** 2 / mse)


def assert_sse_close(gpu_sse: float, ref_sse: float, n: int):
    ref_mse, gpu_mse = ref_sse / n, gpu_sse / n
    if ref_mse < 1e-10:
        assert gpu_mse <= 1e-6, (gpu_mse, ref_mse)
        return
    d = abs(psnr(gpu_mse) - psnr(ref_mse))
    assert d <= PSNR_TOL_DB, (gpu_sse, ref_sse, d)


def assert_coef_close(gpu: np.ndarray, ref: np.ndarray, blocks_norm: np.ndarray):
    """gpu, ref: [nblocks, 64]; blocks_norm: [nblocks] pixel-domain 2-norms."""
    floor = (blocks_norm / 8.0)[:, None]
    bound = COEF_RTOL * np.maximum(np.abs(ref), floor) + 1e-6
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), (np.argwhere(bad)[:5], gpu[bad][:5], ref[bad][:5])


def assert_u8_close(gpu: np.ndarray, ref_u8: np.ndarray, ref_x: np.ndarray, tie_window: float):
    d = np.abs(gpu.astype(np.int32) - ref_u8.astype(np.int32))
    assert d.max() <= 1, int(d.max())
    frac = np.abs(ref_x - np.floor(ref_x) - 0.5)
    inside = (ref_x > -0.5 - tie_window) & (ref_x < 255.5 + tie_window)
    strict = ~((frac < tie_window) & inside)
    mism = (d > 0) & strict
    assert not mism.any(), (np.argwhere(mism)[:5], ref_x[mism][:5])


def block_norms(img: np.ndarray) -> np.ndarray:
    h, w = img.shape
    b = img.astype(np.float64).reshape(h // 8, 8, w // 8, 8).transpose(0, 2, 1, 3).reshape(-1, 64)
    return np.sqrt((b ** 2).sum(axis=1))


def pageable_direct_supported() -> bool:
    """Whether the current device reads and writes pageable host memory through the host's page tables
    (cudaDevAttrPageableMemoryAccess = 88 and cudaDevAttrPageableMemoryAccessUsesHostPageTables = 100, asked
    of the CUDA runtime directly)."""
    import ctypes
    import glob
    import os
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        for c in sorted(glob.glob(os.path.join(d, "lib64", "libcudart.so*"))) if d else []:
            try:
                rt = ctypes.CDLL(c)
            except OSError:
                continue
            dev, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            if rt.cudaGetDevice(ctypes.byref(dev)) != 0:
                return False
            if rt.cudaDeviceGetAttribute(ctypes.byref(a), 88, dev) != 0:
                return False
            if rt.cudaDeviceGetAttribute(ctypes.byref(b), 100, dev) != 0:
                return False
            return a.value == 1 and b.value == 1
    return False
