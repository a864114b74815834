"""Seeded synthetic inputs shared by the tests, the benchmark and the examples.

This module holds no arithmetic of the compression method: it only makes
uint8 planes.  Natural greyscale images have power spectra that fall off
roughly as 1/f^2, so the paper's 512x512 8-bit test images (Sec. 3; the
image bank itself is not available here) are stood in for by Gaussian noise
shaped to a 1/f^alpha power spectrum and min-max scaled to [0, 255].

Recipe (``image_1f``):
  1. z ~ N(0, 1)^(h x w) from numpy's PCG64 seeded with ``seed``;
  2. Z = FFT2(z) * |f|^(-alpha/2), f = hypot(fftfreq(h), fftfreq(w)), gain 0 at f = 0;
  3. x = Re IFFT2(Z);
  4. u8 = rint(255 (x - min x) / (max x - min x)).
alpha = 2 for luma / greyscale, alpha = 3 for the smoother chroma planes.

Large workloads (4K video, thousands of uneven images, serving traces) are
built from a small pool of such fields so that they can be generated on the
device in seconds; see ``video_yuv420`` and ``uneven_batch``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _shaped_noise(h: int, w: int, alpha: float, rng: np.random.Generator) -> np.ndarray:
    z = rng.standard_normal((h, w))
    f = np.hypot(np.fft.fftfreq(h)[:, None], np.fft.fftfreq(w)[None, :])
    gain = np.zeros_like(f)
    nz = f > 0
    gain[nz] = f[nz] ** (-alpha / 2.0)
    return np.real(np.fft.ifft2(np.fft.fft2(z) * gain))


def _to_u8(x: np.ndarray) -> np.ndarray:
    lo, hi = float(x.min()), float(x.max())
    if hi <= lo:
        return np.zeros(x.shape, dtype=np.uint8)
    return np.rint(255.0 * (x - lo) / (hi - lo)).astype(np.uint8)


def image_1f(h: int, w: int, alpha: float = 2.0, seed: int = 0) -> np.ndarray:
    """One seeded 1/f^alpha uint8 plane of shape (h, w)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _to_u8(_shaped_noise(h, w, alpha, rng))


def image_batch(n: int, h: int = 512, w: int = 512, alpha: float = 2.0, seed0: int = 0) -> np.ndarray:
    """n images with seeds seed0 .. seed0+n-1; uint8 [n, h, w]."""
    return np.stack([image_1f(h, w, alpha, seed0 + i) for i in range(n)])


def random_bytes(shape, seed: int = 0) -> np.ndarray:
    """Uniform random uint8 (worst case for the transform: no spectral decay)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 256, size=shape, dtype=np.uint8)


# --------------------------------------------------------------------- video

def _field_pool(n: int, h: int, w: int, alpha: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n, h, w), dtype=np.float32)
    for i in range(n):
        x = _shaped_noise(h, w, alpha, rng)
        out[i] = (x / x.std()).astype(np.float32)
    return out


def video_yuv420(n_frames: int, height: int = 2160, width: int = 3840, seed: int = 0, rho: float = 0.98,
                 pool: int = 8, device: str = "cpu"):
    """A drifting synthetic YUV 4:2:0 clip as three torch uint8 tensors.

    Y is [n, height, width] (alpha = 2), U and V are [n, height/2, width/2]
    (alpha = 3).  Per plane kind the noise field follows
    z_t = rho z_{t-1} + sqrt(1 - rho^2) e_t, where e_t is a pool field
    circularly shifted by a seeded random offset (a shift of a stationary
    1/f field is again such a field), and every frame is scaled by the
    min/max of frame 0 and clamped, so frames stay comparable.
    """
    import torch

    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    planes = []
    for kind, (h, w, alpha) in enumerate(((height, width, 2.0), (height // 2, width // 2, 3.0),
                                          (height // 2, width // 2, 3.0))):
        base = torch.from_numpy(_field_pool(pool, h, w, alpha, seed * 3 + kind)).to(device)
        out = torch.empty((n_frames, h, w), dtype=torch.uint8, device=device)
        z = base[0].clone()
        lo, hi = float(z.min()), float(z.max())
        scale = 255.0 / (hi - lo)
        c = math.sqrt(1.0 - rho * rho)
        for t in range(n_frames):
            if t > 0:
                dy, dx = int(rng.integers(0, h)), int(rng.integers(0, w))
                e = torch.roll(base[t % pool], shifts=(dy, dx), dims=(0, 1))
                z.mul_(rho).add_(e, alpha=c)
            out[t] = ((z - lo) * scale).round_().clamp_(0, 255).to(torch.uint8)
        planes.append(out)
    return planes


# ------------------------------------------------------------- uneven batches

@dataclass
class ImageSpec:
    """Shape and retained-coefficient count of one image of an uneven batch."""
    w: int
    h: int
    planes: int
    r: int


def uneven_specs(n: int, seed: int = 0, lo: int = 64, hi: int = 2048, rs=(4, 10, 16, 32)) -> list[ImageSpec]:
    """Widths and heights uniform over multiples of 8 in [lo, hi], 1 or 3 planes, r from ``rs``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.arange(lo, hi + 1, 8)
    out = []
    for _ in range(n):
        out.append(ImageSpec(int(rng.choice(sides)), int(rng.choice(sides)), int(rng.choice([1, 3])),
                             int(rng.choice(rs))))
    return out


def crop_pool(pool_side: int = 2048, n: int = 4, seed: int = 0, alpha: float = 2.0) -> np.ndarray:
    """Pool of 1/f^alpha float fields from which uneven-batch planes are cropped."""
    return _field_pool(n, pool_side, pool_side, alpha, seed)


def crop_plane(pool: np.ndarray, h: int, w: int, rng: np.random.Generator) -> np.ndarray:
    """A uint8 plane: a circular crop of a random pool field at a random offset, min-max scaled."""
    k = int(rng.integers(0, pool.shape[0]))
    dy, dx = int(rng.integers(0, pool.shape[1])), int(rng.integers(0, pool.shape[2]))
    ys = (np.arange(h) + dy) % pool.shape[1]
    xs = (np.arange(w) + dx) % pool.shape[2]
    return _to_u8(pool[k][np.ix_(ys, xs)].astype(np.float64))


# ------------------------------------------------------------------ serving

@dataclass
class Request:
    """One serving request: arrival time (s), square side, planes, r."""
    t: float
    side: int
    planes: int
    r: int


def poisson_trace(rate: float, n: int, seed: int = 0, lo: int = 256, hi: int = 4096) -> list[Request]:
    """Poisson arrivals at ``rate`` req/s; side = 8 round(exp(U(ln lo, ln hi)) / 8); 1 or 3 planes; r ~ U{1..64}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        side = int(8 * round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 8))
        out.append(Request(t, side, int(rng.choice([1, 3])), int(rng.integers(1, 65))))
    return out


def field_u8_torch(h: int, w: int, alpha: float, seed: int, device: str = "cpu", planes: int = 1):
    """[planes, h, w] uint8 1/f^alpha planes generated with torch on `device` (same recipe as
    image_1f, torch's generator instead of numpy's; used for large pools)."""
    import torch

    g = torch.Generator(device="cpu").manual_seed(seed)
    out = torch.empty((planes, h, w), dtype=torch.uint8, device=device)
    fy = torch.fft.fftfreq(h, device=device)[:, None]
    fx = torch.fft.fftfreq(w, device=device)[None, :]
    f = torch.hypot(fy, fx)
    gain = torch.where(f > 0, f.clamp_min(1e-12) ** (-alpha / 2.0), torch.zeros_like(f))
    for p in range(planes):
        z = torch.randn((h, w), generator=g).to(device)
        x = torch.fft.ifft2(torch.fft.fft2(z) * gain).real
        lo, hi = x.min(), x.max()
        out[p] = torch.round(255.0 * (x - lo) / (hi - lo)).to(torch.uint8)
    return out
