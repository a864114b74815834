"""Thin ctypes binding of librdct (include/rdct.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  torch is used for device memory and streams.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import build_lib

KIND_RDCT = 0
KIND_DCT = 1
# other transforms of the paper (rdct_variant)
VARIANT_ROUND, VARIANT_CEIL, VARIANT_FLOOR, VARIANT_SDCT, VARIANT_SDCT_POLAR = 0, 1, 2, 3, 4
VARIANTS = {"round": 0, "ceil": 1, "floor": 2, "sdct": 3, "sdct_polar": 4}

_STATUS = {0: "ok", 1: "invalid argument", 2: "invalid shape", 3: "out of memory", 4: "too large",
           5: "CUDA error", 6: "timeout", 7: "busy", 8: "not found", 9: "cancelled"}


class RdctError(RuntimeError):
    """A librdct call returned a status other than RDCT_OK."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Plane(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("pitch", ctypes.c_int64), ("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class Out(ctypes.Structure):
    _fields_ = [("u8", ctypes.c_void_p), ("f32", ctypes.c_void_p), ("pitch", ctypes.c_int64),
                ("pitch_f32", ctypes.c_int64)]


class Job(ctypes.Structure):
    _fields_ = [("src", Plane), ("dst", ctypes.c_void_p), ("dst_pitch", ctypes.c_int64), ("r", ctypes.c_int32),
                ("image", ctypes.c_int32)]


class Tune(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("items_per_chunk", ctypes.c_int32), ("blocks_per_thread", ctypes.c_int32),
                ("staging", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class HostJob(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("pitch", ctypes.c_int64),
                ("w", ctypes.c_int32), ("h", ctypes.c_int32), ("r", ctypes.c_int32), ("image", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("streams", ctypes.c_int32), ("max_wait_us", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("pitch", ctypes.c_int64),
                ("plane_stride", ctypes.c_int64), ("w", ctypes.c_int32), ("h", ctypes.c_int32),
                ("planes", ctypes.c_int32), ("r", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sse", ctypes.c_double), ("mse", ctypes.c_double),
                ("psnr", ctypes.c_double), ("latency_us", ctypes.c_double), ("sse_u8", ctypes.c_double),
                ("mse_u8", ctypes.c_double), ("psnr_u8", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "status"}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("gpixels_per_s", ctypes.c_double),
                ("peak_resident_bytes", ctypes.c_int64), ("p999_us", ctypes.c_double)]


_lib = None
_lock = threading.Lock()

# name -> (argtypes) ; all return rdct_status (int) unless listed in _RESTYPE
_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "rdct_status_string": [ctypes.c_int],
    "rdct_last_error": [ctypes.c_char_p, ctypes.c_size_t],
    "rdct_version": [],
    "rdct_sync": [_vp],
    "rdct_forward": [ctypes.POINTER(Plane), _vp, _vp],
    "rdct_forward_f32": [ctypes.POINTER(Plane), ctypes.c_int, _vp, _vp],
    "rdct_compress": [_vp, _i64, _i32, _vp, _vp],
    "rdct_inverse": [_vp, _i64, _i64, _i32, ctypes.c_int, ctypes.POINTER(Out), _vp],
    "rdct_mse_psnr": [ctypes.POINTER(Plane), ctypes.POINTER(Out), _vp, _vp, _vp],
    "rdct_fused": [ctypes.POINTER(Plane), _i32, ctypes.c_int, ctypes.POINTER(Out), _vp, _vp, _vp],
    "rdct_uqi": [ctypes.POINTER(Plane), ctypes.POINTER(Out), _vp, _vp],
    "rdct_variant_matrices": [ctypes.c_int, _vp, _vp],
    "rdct_pipeline_set_mode": [_vp, _i32],
    "rdct_spectral_error": [ctypes.c_int, _i32, _vp, _vp],
    "rdct_fused_variant": [ctypes.POINTER(Plane), _i32, ctypes.c_int, ctypes.POINTER(Out), _vp, _vp],
    "rdct_sweep": [ctypes.POINTER(Plane), _i32, ctypes.c_int, _vp, _vp],
    "rdct_sweep_noalloc": [ctypes.POINTER(Plane), _i32, ctypes.c_int, _vp, _vp],
    "rdct_batch_plan_create": [ctypes.POINTER(Job), _i32, _i32, ctypes.POINTER(Tune), ctypes.POINTER(_vp)],
    "rdct_batch_run": [_vp, _vp, _vp, _vp],
    "rdct_batch_run_per_plane": [_vp, _vp, _vp, _vp],
    "rdct_batch_plan_get_tune": [_vp, ctypes.POINTER(Tune)],
    "rdct_batch_plan_kernels": [_vp, ctypes.POINTER(_i32)],
    "rdct_batch_plan_destroy": [_vp],
    "rdct_autotune": [ctypes.POINTER(Job), _i32, _i32, ctypes.POINTER(Tune), _vp],
    "rdct_autotune_cache_save": [ctypes.c_char_p],
    "rdct_autotune_cache_load": [ctypes.c_char_p, ctypes.POINTER(_i32)],
    "rdct_autotune_cache_clear": [],
    "rdct_pipeline_create": [_i64, _i32, ctypes.POINTER(_vp)],
    "rdct_pipeline_run": [_vp, ctypes.POINTER(HostJob), _i32, _i32, _vp, _vp],
    "rdct_pipeline_destroy": [_vp],
    "rdct_server_create": [ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)],
    "rdct_server_submit": [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
    "rdct_server_wait": [_vp, ctypes.c_uint64, _i64, ctypes.POINTER(Result)],
    "rdct_server_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(Result)],
    "rdct_server_cancel": [_vp, ctypes.c_uint64],
    "rdct_server_stats_get": [_vp, ctypes.POINTER(ServerStats)],
    "rdct_server_destroy": [_vp],
    "rdct_server_inject_alloc_failures": [_vp, _i32],
    "rdct_arena_create": [_i64, _i64, ctypes.POINTER(_vp)],
    "rdct_arena_alloc": [_vp, _i64, ctypes.POINTER(_i64)],
    "rdct_arena_free": [_vp, _i64],
    "rdct_arena_used": [_vp],
    "rdct_arena_largest_free": [_vp],
    "rdct_arena_destroy": [_vp],
}
_RESTYPE = {"rdct_status_string": ctypes.c_char_p, "rdct_last_error": ctypes.c_size_t, "rdct_version": ctypes.c_int32,
            "rdct_arena_used": ctypes.c_int64, "rdct_arena_largest_free": ctypes.c_int64}


def lib_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = True):
    """Load librdct.so (building it first if asked); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"librdct is not built ({path}); run build_lib.build()")
            build_lib.build()
        lib = ctypes.CDLL(path)
        for name, argt in _SIGS.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.argtypes = argt
            fn.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = lib
        return lib


def exported_names() -> list[str]:
    lib = load()
    return [n for n in _SIGS if getattr(lib, n, None) is not None]


def sync(stream=None) -> None:
    """rdct_sync: wait for the work on `stream` and raise on an asynchronous error (RdctError)."""
    _check(load().rdct_sync(_stream(stream)), "rdct_sync")


def _check(status: int, what: str):
    if status != 0:
        lib = load()
        buf = ctypes.create_string_buffer(1024)
        lib.rdct_last_error(buf, 1024)
        raise RdctError(status, f"{what}: {buf.value.decode(errors='replace')}")


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")


def plane_of(t: torch.Tensor) -> Plane:
    """A 2-D uint8 CUDA tensor (rows may be padded: stride(1) must be 1) as an rdct_plane."""
    _require_cuda(t, "plane", torch.uint8)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("plane must be a 2-D uint8 tensor with unit column stride")
    return Plane(t.data_ptr(), t.stride(0), t.shape[1], t.shape[0])


# ------------------------------------------------------------------- steps

def forward(img: torch.Tensor, stream=None) -> torch.Tensor:
    """Y = C0 A C0^T per 8x8 block; int32 [h/8, w/8, 8, 8]."""
    p = plane_of(img)
    Y = torch.empty((p.h // 8, p.w // 8, 8, 8), dtype=torch.int32, device=img.device)
    _check(load().rdct_forward(ctypes.byref(p), Y.data_ptr(), _stream(stream)), "rdct_forward")
    return Y


def forward_f32(img: torch.Tensor, kind: int = KIND_RDCT, stream=None) -> torch.Tensor:
    """Orthonormal coefficients (S Y S or the exact DCT) in FP32; [h/8, w/8, 8, 8]."""
    p = plane_of(img)
    Y = torch.empty((p.h // 8, p.w // 8, 8, 8), dtype=torch.float32, device=img.device)
    _check(load().rdct_forward_f32(ctypes.byref(p), kind, Y.data_ptr(), _stream(stream)), "rdct_forward_f32")
    return Y


def compress(Y: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    """First r zigzag coefficients of S Y S per block; FP32 [nblocks, r]."""
    _require_cuda(Y, "Y", torch.int32)
    Y = Y.contiguous()
    nb = Y.numel() // 64
    Yc = torch.empty((nb, r), dtype=torch.float32, device=Y.device)
    _check(load().rdct_compress(Y.data_ptr(), nb, r, Yc.data_ptr(), _stream(stream)), "rdct_compress")
    return Yc


def inverse(Yc: torch.Tensor, nbw: int, nbh: int, r: int, kind: int = KIND_RDCT, want_u8: bool = True,
            want_f32: bool = False, stream=None):
    """Reconstruct from packed coefficients; returns (u8 or None, f32 or None)."""
    _require_cuda(Yc, "Yc", torch.float32)
    Yc = Yc.contiguous()
    dev = Yc.device
    u8 = torch.empty((nbh * 8, nbw * 8), dtype=torch.uint8, device=dev) if want_u8 else None
    f32 = torch.empty((nbh * 8, nbw * 8), dtype=torch.float32, device=dev) if want_f32 else None
    out = Out(u8.data_ptr() if u8 is not None else None, f32.data_ptr() if f32 is not None else None, nbw * 8, nbw * 8)
    _check(load().rdct_inverse(Yc.data_ptr(), nbw, nbh, r, kind, ctypes.byref(out), _stream(stream)), "rdct_inverse")
    return u8, f32


def mse_psnr(ref: torch.Tensor, rec: torch.Tensor, stream=None):
    """(MSE, PSNR) of rec (uint8 or float32 plane) against ref, as device float64 scalars."""
    p = plane_of(ref)
    _require_cuda(rec, "rec")
    if rec.dim() != 2 or tuple(rec.shape) != tuple(ref.shape) or rec.stride(1) != 1:
        raise ValueError("rec must be a 2-D plane of ref's shape with unit column stride")
    if rec.dtype == torch.uint8:
        out = Out(rec.data_ptr(), None, rec.stride(0), 0)
    elif rec.dtype == torch.float32:
        out = Out(None, rec.data_ptr(), 0, rec.stride(0))
    else:
        raise ValueError("rec must be uint8 or float32")
    res = torch.empty(2, dtype=torch.float64, device=ref.device)
    _check(load().rdct_mse_psnr(ctypes.byref(p), ctypes.byref(out), res.data_ptr(), res.data_ptr() + 8,
                                _stream(stream)), "rdct_mse_psnr")
    return res[0], res[1]


def uqi(ref: torch.Tensor, rec: torch.Tensor, stream=None) -> torch.Tensor:
    """Universal quality index of rec (uint8 or float32 plane) against ref; device float64 scalar."""
    p = plane_of(ref)
    _require_cuda(rec, "rec")
    if rec.dim() != 2 or tuple(rec.shape) != tuple(ref.shape) or rec.stride(1) != 1:
        raise ValueError("rec must be a 2-D plane of ref's shape with unit column stride")
    if rec.dtype == torch.uint8:
        out = Out(rec.data_ptr(), None, rec.stride(0), 0)
    elif rec.dtype == torch.float32:
        out = Out(None, rec.data_ptr(), 0, rec.stride(0))
    else:
        raise ValueError("rec must be uint8 or float32")
    q = torch.empty(1, dtype=torch.float64, device=ref.device)
    _check(load().rdct_uqi(ctypes.byref(p), ctypes.byref(out), q.data_ptr(), _stream(stream)), "rdct_uqi")
    return q[0]


def variant_matrices(variant: int):
    """(F, G) of a variant as float64 numpy arrays [8, 8], computed by the library on the host."""
    import numpy as np
    F = np.zeros(64)
    G = np.zeros(64)
    _check(load().rdct_variant_matrices(variant, F.ctypes.data, G.ctypes.data), "rdct_variant_matrices")
    return F.reshape(8, 8), G.reshape(8, 8)


def spectral_error(variant: int, npoints: int = 20001, want_curves: bool = False):
    """(eps [8], D [8, npoints] or None, omega [npoints]) of Sec. 2 for a variant's forward matrix (host)."""
    import numpy as np
    eps = np.zeros(8)
    D = np.zeros((8, npoints)) if want_curves else None
    _check(load().rdct_spectral_error(variant, npoints, D.ctypes.data if D is not None else None, eps.ctypes.data),
           "rdct_spectral_error")
    return eps, D, np.linspace(0.0, np.pi, npoints)


def fused_variant(img: torch.Tensor, r: int, variant: int, want_u8: bool = True, want_f32: bool = False,
                  sse: torch.Tensor | None = None, stream=None):
    """Block experiment with another transform (signed DCT, ceil/floor variants); returns (u8, f32, sse[1])."""
    p = plane_of(img)
    dev = img.device
    u8 = torch.empty((p.h, p.w), dtype=torch.uint8, device=dev) if want_u8 else None
    f32 = torch.empty((p.h, p.w), dtype=torch.float32, device=dev) if want_f32 else None
    if sse is None:
        sse = torch.empty(1, dtype=torch.float64, device=dev)
    out = Out(u8.data_ptr() if u8 is not None else None, f32.data_ptr() if f32 is not None else None,
              u8.stride(0) if u8 is not None else 0, p.w)
    _check(load().rdct_fused_variant(ctypes.byref(p), r, variant, ctypes.byref(out), sse.data_ptr(),
                                     _stream(stream)), "rdct_fused_variant")
    return u8, f32, sse


def fused(img: torch.Tensor, r: int, kind: int = KIND_RDCT, want_u8: bool = True, want_f32: bool = False,
          out_u8: torch.Tensor | None = None, sse: torch.Tensor | None = None, sse_u8: torch.Tensor | None = None,
          stream=None):
    """Forward + keep r + inverse + SSE in one kernel; returns (u8 or None, f32 or None, sse [1] float64).
    sse_u8 (a float64 CUDA tensor of one element, or None) receives the squared error of the 8-bit
    reconstruction."""
    p = plane_of(img)
    dev = img.device
    u8 = out_u8 if out_u8 is not None else (torch.empty((p.h, p.w), dtype=torch.uint8, device=dev) if want_u8 else None)
    f32 = torch.empty((p.h, p.w), dtype=torch.float32, device=dev) if want_f32 else None
    if sse is None:
        sse = torch.empty(1, dtype=torch.float64, device=dev)
    if sse_u8 is not None:
        _require_cuda(sse_u8, "sse_u8", torch.float64)
    out = Out(u8.data_ptr() if u8 is not None else None, f32.data_ptr() if f32 is not None else None,
              u8.stride(0) if u8 is not None else 0, p.w)
    _check(load().rdct_fused(ctypes.byref(p), r, kind, ctypes.byref(out), sse.data_ptr(),
                             sse_u8.data_ptr() if sse_u8 is not None else None, _stream(stream)), "rdct_fused")
    return u8, f32, sse


def sweep(planes, kind: int = KIND_RDCT, stream=None) -> torch.Tensor:
    """SSE(r) for r = 1..64 per plane; float64 [n, 64].  planes: [n, h, w] uint8 tensor or list of 2-D tensors."""
    if isinstance(planes, torch.Tensor) and planes.dim() == 3:
        planes = list(planes.unbind(0))
    arr = (Plane * len(planes))(*[plane_of(t) for t in planes])
    dev = planes[0].device
    out = torch.empty((len(planes), 64), dtype=torch.float64, device=dev)
    _check(load().rdct_sweep(arr, len(planes), kind, out.data_ptr(), _stream(stream)), "rdct_sweep")
    return out


def sweep_noalloc(planes, out: torch.Tensor, kind: int = KIND_RDCT, stream=None) -> torch.Tensor:
    """rdct_sweep without allocation inside the library, for callers that cannot allocate device
    memory at call time.  ``out`` is a caller-owned float64 [n, 64] CUDA tensor (allocated in
    advance).  At most 2048 planes / about 1.07 Gpixel per call; concurrent calls race on the
    library's fixed table storage and must be serialised by the caller."""
    arr = planes if isinstance(planes, ctypes.Array) else plane_array(planes)
    _require_cuda(out, "out", torch.float64)
    if out.shape != (len(arr), 64) or not out.is_contiguous():
        raise ValueError("out must be a contiguous [n, 64] float64 tensor")
    _check(load().rdct_sweep_noalloc(arr, len(arr), kind, out.data_ptr(), _stream(stream)), "rdct_sweep_noalloc")
    return out


def plane_array(planes) -> ctypes.Array:
    """rdct_plane[] for a list of 2-D uint8 CUDA tensors or a [n, h, w] tensor (build once, reuse)."""
    if isinstance(planes, torch.Tensor) and planes.dim() == 3:
        planes = list(planes.unbind(0))
    return (Plane * len(planes))(*[plane_of(t) for t in planes])


# ----------------------------------------------------------------- batches

@dataclass
class BatchJob:
    """One plane of a batch (device tensors)."""
    src: torch.Tensor
    dst: torch.Tensor | None
    r: int
    image: int


class BatchPlan:
    """A persistent, graph-captured launch over many uneven planes."""

    def __init__(self, jobs: list[BatchJob], nimages: int, tune: dict | None = None):
        self._keep = [(j.src, j.dst) for j in jobs]
        self.nimages = nimages
        arr = (Job * len(jobs))()
        for i, j in enumerate(jobs):
            arr[i].src = plane_of(j.src)
            arr[i].dst = j.dst.data_ptr() if j.dst is not None else None
            arr[i].dst_pitch = j.dst.stride(0) if j.dst is not None else 0
            arr[i].r = j.r
            arr[i].image = j.image
        self._jobs = arr
        t = None
        if tune is not None:
            t = Tune(tune["warps_per_cta"], tune["ctas_per_sm"], tune["items_per_chunk"],
                     tune.get("blocks_per_thread", 1), tune.get("staging", 0))
        h = ctypes.c_void_p()
        _check(load().rdct_batch_plan_create(arr, len(jobs), nimages, ctypes.byref(t) if t else None, ctypes.byref(h)),
               "rdct_batch_plan_create")
        self._h = h

    @property
    def tune(self) -> dict:
        t = Tune()
        _check(load().rdct_batch_plan_get_tune(self._h, ctypes.byref(t)), "rdct_batch_plan_get_tune")
        return t.as_dict()

    def kernels_per_run(self) -> int:
        """Kernels one run launches (one per non-empty chunk group, plus the error conversion)."""
        k = _i32()
        _check(load().rdct_batch_plan_kernels(self._h, ctypes.byref(k)), "rdct_batch_plan_kernels")
        return int(k.value)

    def run(self, sse: torch.Tensor, stream=None, sse_u8: torch.Tensor | None = None):
        """sse (and sse_u8 if given): float64 CUDA tensors of nimages elements."""
        _check(load().rdct_batch_run(self._h, sse.data_ptr(), sse_u8.data_ptr() if sse_u8 is not None else None,
                                     _stream(stream)), "rdct_batch_run")

    def run_per_plane(self, sse: torch.Tensor, stream=None, sse_u8: torch.Tensor | None = None):
        _check(load().rdct_batch_run_per_plane(self._h, sse.data_ptr(),
                                               sse_u8.data_ptr() if sse_u8 is not None else None, _stream(stream)),
               "rdct_batch_run_per_plane")

    def close(self):
        if self._h:
            load().rdct_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(jobs: list[BatchJob], nimages: int, stream=None) -> dict:
    arr = (Job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i].src = plane_of(j.src)
        arr[i].dst = j.dst.data_ptr() if j.dst is not None else None
        arr[i].dst_pitch = j.dst.stride(0) if j.dst is not None else 0
        arr[i].r = j.r
        arr[i].image = j.image
    t = Tune()
    _check(load().rdct_autotune(arr, len(jobs), nimages, ctypes.byref(t), _stream(stream)), "rdct_autotune")
    return t.as_dict()


def autotune_cache_save(path: str) -> None:
    """rdct_autotune_cache_save: this process's autotune results to `path` (one JSON object per line)."""
    _check(load().rdct_autotune_cache_save(os.fsencode(path)), "rdct_autotune_cache_save")


def autotune_cache_load(path: str) -> int:
    """rdct_autotune_cache_load: merge a saved cache; returns the number of entries taken."""
    n = _i32()
    _check(load().rdct_autotune_cache_load(os.fsencode(path), ctypes.byref(n)), "rdct_autotune_cache_load")
    return n.value


def autotune_cache_clear() -> None:
    """rdct_autotune_cache_clear: forget every autotune result of this process."""
    _check(load().rdct_autotune_cache_clear(), "rdct_autotune_cache_clear")


# ---------------------------------------------------------- host streaming

class Pipeline:
    """Planes in host memory streamed through the fused path (copies overlapped with kernels)."""

    AUTO, STAGED, DIRECT = 0, 1, 2

    def __init__(self, device_budget_bytes: int = 1 << 30, depth: int = 3, mode: int = 0):
        h = ctypes.c_void_p()
        _check(load().rdct_pipeline_create(device_budget_bytes, depth, ctypes.byref(h)), "rdct_pipeline_create")
        self._h = h
        _check(load().rdct_pipeline_set_mode(h, mode), "rdct_pipeline_set_mode")

    def run(self, jobs: list[tuple], nimages: int, want_u8_error: bool = False):
        """jobs: (src, dst or None, r, image) with src/dst 2-D uint8 host arrays (numpy or CPU tensors).
        Returns the per-image SSE list, or (SSE list, 8-bit SSE list) with want_u8_error."""
        arr = (HostJob * len(jobs))()
        keep = []
        for i, (src, dst, r, image) in enumerate(jobs):
            sp, pitch, h, w = _host_ptr(src)
            dp = _host_ptr(dst)[0] if dst is not None else None
            arr[i] = HostJob(sp, dp, pitch, w, h, r, image)
            keep.append((src, dst))
        sse = (ctypes.c_double * max(nimages, 1))()
        sse8 = (ctypes.c_double * max(nimages, 1))() if want_u8_error else None
        _check(load().rdct_pipeline_run(self._h, arr, len(jobs), nimages, sse, sse8), "rdct_pipeline_run")
        if want_u8_error:
            return list(sse[:nimages]), list(sse8[:nimages])
        return list(sse[:nimages])

    def close(self):
        if self._h:
            load().rdct_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(a):
    """(address, pitch, h, w) of a 2-D (or [planes, h, w]) uint8 host array with unit column stride."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.uint8 or a.stride(-1) != 1:
            raise ValueError("host plane must be a CPU uint8 tensor with unit column stride")
        return a.data_ptr(), a.stride(-2), a.shape[-2], a.shape[-1]
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.uint8 or a.strides[-1] != 1:
        raise ValueError("host plane must be a uint8 numpy array with unit column stride")
    return a.ctypes.data, a.strides[-2], a.shape[-2], a.shape[-1]


# ------------------------------------------------------------------ serving

class Server:
    """Continuous-batching server; requests are host images [planes, h, w] (uint8)."""

    def __init__(self, device_budget_bytes: int = 8 << 30, max_batch: int = 64, queue_capacity: int = 4096,
                 streams: int = 2, max_wait_us: int = 0):
        opts = ServerOpts(device_budget_bytes, max_batch, queue_capacity, streams, max_wait_us)
        h = ctypes.c_void_p()
        _check(load().rdct_server_create(ctypes.byref(opts), ctypes.byref(h)), "rdct_server_create")
        self._h = h
        self._keep = {}

    def submit(self, src, r: int, dst=None) -> int:
        """Queue an image; src/dst are host uint8 arrays [planes, h, w] (strided views allowed; dst must
        have the same strides as src)."""
        if src.ndim == 2:
            src = src[None]
            dst = dst[None] if dst is not None else None
        sp, pitch, h, w = _host_ptr(src)
        stride = src.stride(0) if isinstance(src, torch.Tensor) else src.strides[0]
        dp = None
        if dst is not None:
            dp, dpitch, _, _ = _host_ptr(dst)
            dstride = dst.stride(0) if isinstance(dst, torch.Tensor) else dst.strides[0]
            if dpitch != pitch or (src.shape[0] > 1 and dstride != stride):
                raise ValueError("dst must have the same row pitch and plane stride as src")
        req = Request(sp, dp, pitch, stride if src.shape[0] > 1 else 0, w, h, src.shape[0], r)
        t = ctypes.c_uint64()
        _check(load().rdct_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "rdct_server_submit")
        self._keep[t.value] = (src, dst)
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        res = Result()
        st = load().rdct_server_wait(self._h, ticket, timeout_us, ctypes.byref(res))
        if st != 6:  # keep buffers alive while still pending
            self._keep.pop(ticket, None)
        _check(st, "rdct_server_wait")
        return res.as_dict()

    def poll(self, ticket: int):
        res = Result()
        st = load().rdct_server_poll(self._h, ticket, ctypes.byref(res))
        if st == 7:
            return None
        self._keep.pop(ticket, None)
        _check(st, "rdct_server_poll")
        return res.as_dict()

    def cancel(self, ticket: int):
        _check(load().rdct_server_cancel(self._h, ticket), "rdct_server_cancel")

    def inject_alloc_failures(self, n: int):
        _check(load().rdct_server_inject_alloc_failures(self._h, n), "rdct_server_inject_alloc_failures")

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().rdct_server_stats_get(self._h, ctypes.byref(st)), "rdct_server_stats_get")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            _check(load().rdct_server_destroy(self._h), "rdct_server_destroy")
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Arena:
    """The server's offset sub-allocator (host logic only; usable without a GPU)."""

    def __init__(self, size: int, align: int = 256):
        h = ctypes.c_void_p()
        _check(load().rdct_arena_create(size, align, ctypes.byref(h)), "rdct_arena_create")
        self._h = h

    def alloc(self, nbytes: int):
        off = ctypes.c_int64()
        st = load().rdct_arena_alloc(self._h, nbytes, ctypes.byref(off))
        if st == 3:
            return None
        _check(st, "rdct_arena_alloc")
        return off.value

    def free(self, off: int):
        _check(load().rdct_arena_free(self._h, off), "rdct_arena_free")

    @property
    def used(self) -> int:
        return load().rdct_arena_used(self._h)

    @property
    def largest_free(self) -> int:
        return load().rdct_arena_largest_free(self._h)

    def close(self):
        if self._h:
            load().rdct_arena_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
