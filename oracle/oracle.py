"""FP64 CPU oracle for the RDCT path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this module.  The CUDA library and its Python
binding never import it; the two sides share no code.

This module compiles ``rdct_oracle.c`` (plain FP64 matrix products written
from Sec. 2-3 of Cintra & Bayer, "A DCT Approximation for Image Compression")
and wraps it with numpy.  It also holds the paper's spectral analysis (the
transfer functions H_m, the error D_m and the error energy eps_m of Sec. 2,
Table 2), the quality measures of Sec. 3 (MSE, PSNR, their averages over
images, the absolute percentage error against the exact DCT, the UQI) and the
matrices of the other transforms the paper names (the signed DCT of Sec. 3 and
the floor / ceiling generalisations of its conclusion).

Parity status: every function below is pinned by a test in
``tests/test_oracle_pins.py`` against something other than itself (printed
matrices, Table 2, closed forms, scipy's DCT, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rdct_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librdct_oracle.so")

KIND_RDCT = 0  # C_orth = S C0, the proposed approximation (Sec. 2)
KIND_DCT = 1   # exact orthonormal DCT-II (the comparison baseline of Sec. 3)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        ip = ctypes.POINTER(ctypes.c_int)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_dct_matrix.argtypes = [dp]
        lib.oracle_round_off_matrix.argtypes = [dp]
        lib.oracle_matlab_round.argtypes = [ctypes.c_double]
        lib.oracle_matlab_round.restype = ctypes.c_double
        lib.oracle_orthogonalizer.argtypes = [dp, dp]
        lib.oracle_orth_matrix.argtypes = [dp]
        lib.oracle_zigzag.argtypes = [ip]
        lib.rdct_ref_forward.argtypes = [u8p, i64, i32, i32, i32p]
        lib.rdct_ref_forward_f64.argtypes = [u8p, i64, i32, i32, i32, dp]
        lib.rdct_ref_compress.argtypes = [i32p, i64, i32, dp]
        lib.rdct_ref_inverse.argtypes = [dp, i64, i64, i32, i32, dp, i64]
        lib.rdct_ref_fused.argtypes = [u8p, i64, i32, i32, i32, i32, dp, u8p, dp, dp, i32]
        lib.rdct_ref_sweep.argtypes = [u8p, i64, i32, i32, i32, dp, i32]
        lib.rdct_ref_sse.argtypes = [u8p, i64, i32, i32, u8p, dp, i64, dp]
        lib.rdct_ref_max_threads.argtypes = []
        lib.rdct_ref_uqi.argtypes = [u8p, i64, i32, i32, u8p, dp, i64, i32, dp]
        lib.rdct_ref_fused_general.argtypes = [u8p, i64, i32, i32, i32, dp, dp, dp, u8p, dp, dp, i32]
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(status: int, what: str):
    if status != 0:
        raise RuntimeError(f"oracle {what} failed with status {status}")


def _plane(img: np.ndarray):
    img = np.asarray(img)
    if img.dtype != np.uint8 or img.ndim != 2:
        raise ValueError("a plane is a 2-D uint8 array")
    if img.strides[1] != 1:
        img = np.ascontiguousarray(img)
    h, w = img.shape
    return img, int(img.strides[0]), w, h


# ------------------------------------------------------------------ matrices

def dct_matrix() -> np.ndarray:
    """Sec. 2: the orthonormal 8-point DCT-II matrix C."""
    out = np.zeros(64)
    _load().oracle_dct_matrix(_ptr(out, ctypes.c_double))
    return out.reshape(8, 8)


def matlab_round(v: float) -> float:
    """Sec. 2: Matlab's round (half away from zero)."""
    return _load().oracle_matlab_round(float(v))


def round_off_matrix() -> np.ndarray:
    """Sec. 2: C0 = [2C]."""
    out = np.zeros(64)
    _load().oracle_round_off_matrix(_ptr(out, ctypes.c_double))
    return out.reshape(8, 8)


def orthogonalizer(C0: np.ndarray) -> np.ndarray:
    """Sec. 2: S = sqrt((C0 C0^T)^-1) (diagonal case); raises if C0 C0^T is not diagonal."""
    c0 = np.ascontiguousarray(C0, dtype=np.float64).reshape(64)
    out = np.zeros(64)
    _check(_load().oracle_orthogonalizer(_ptr(c0, ctypes.c_double), _ptr(out, ctypes.c_double)), "orthogonalizer")
    return out.reshape(8, 8)


def orth_matrix() -> np.ndarray:
    """Sec. 2: C_orth = S C0."""
    out = np.zeros(64)
    _check(_load().oracle_orth_matrix(_ptr(out, ctypes.c_double)), "orth_matrix")
    return out.reshape(8, 8)


def zigzag() -> np.ndarray:
    """Sec. 3: zz[k] = row*8+col of the k-th coefficient of the zigzag sequence."""
    out = np.zeros(64, dtype=np.intc)
    _load().oracle_zigzag(_ptr(out, ctypes.c_int))
    return out.astype(np.int64)


def sdct_matrix() -> np.ndarray:
    """The signed DCT of the comparison in Sec. 2 (Table 2), read as sign(C)/sqrt(8)."""
    return np.sign(dct_matrix()) / np.sqrt(8.0)


# ---------------------------------------------------------- other transforms

VARIANTS = ("round", "ceil", "floor", "sdct", "sdct_polar")


def variant_matrices(name: str):
    """(F, G) for the 2-D experiment of Sec. 3: a block A goes to F A F^T and comes back as G Yhat G^T.

    round      -- C_orth of Sec. 2: [2C] with round-off, times (C0 C0^T)^(-1/2); G = F^T.
    ceil/floor -- the conclusion's generalisations: ceil(2C) / floor(2C) in place of [2C], orthogonalised the
                  same way (polar factor (T T^T)^(-1/2) T); floor(2C) has a zero first row, so T T^T is singular
                  and no such factor exists (ValueError).
    sdct       -- the signed DCT compared in Sec. 3, sign(C) / sqrt(8) (the scaling of Table 2), rebuilt with
                  its exact inverse G = F^(-1).
    sdct_polar -- sign(C) orthogonalised like C0; G = F^T.
    """
    C = dct_matrix()
    if name == "round":
        T = round_off_matrix()
    elif name == "ceil":
        T = np.ceil(2.0 * C)
    elif name == "floor":
        T = np.floor(2.0 * C)
    elif name in ("sdct", "sdct_polar"):
        T = np.sign(C)
    else:
        raise ValueError(f"unknown variant {name!r}")
    if name == "sdct":
        F = T / np.sqrt(8.0)
        return F, np.linalg.inv(F)
    gram = T @ T.T
    lam, V = np.linalg.eigh(gram)
    if lam.min() <= 1e-9 * lam.max():
        raise ValueError(f"variant {name!r}: T T^T is singular, no orthogonal polar factor")
    S = V @ np.diag(lam ** -0.5) @ V.T
    F = S @ T
    return F, F.T


def fused_general(img: np.ndarray, r: int, F: np.ndarray, G: np.ndarray, want_xhat: bool = True,
                  want_u8: bool = True, nthreads: int = 0):
    """Sec. 3 with Y = F A F^T and X = G Yhat G^T; returns (xhat or None, u8 or None, sse, sse_u8)."""
    img, pitch, w, h = _plane(img)
    F = np.ascontiguousarray(F, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    xhat = np.zeros((h, w)) if want_xhat else None
    u8 = np.zeros((h, w), dtype=np.uint8) if want_u8 else None
    sse = np.zeros(1)
    sse_u8 = np.zeros(1)
    _check(_load().rdct_ref_fused_general(_ptr(img, ctypes.c_uint8), pitch, w, h, r, _ptr(F, ctypes.c_double),
                                          _ptr(G, ctypes.c_double),
                                          _ptr(xhat, ctypes.c_double) if xhat is not None else None,
                                          _ptr(u8, ctypes.c_uint8) if u8 is not None else None,
                                          _ptr(sse, ctypes.c_double), _ptr(sse_u8, ctypes.c_double), nthreads),
           "fused_general")
    return xhat, u8, float(sse[0]), float(sse_u8[0])


# ------------------------------------------------------------- block pipeline

def forward(img: np.ndarray) -> np.ndarray:
    """Integer Y = C0 A C0^T per 8x8 block; returns int32 [nbh, nbw, 8, 8]."""
    img, pitch, w, h = _plane(img)
    Y = np.zeros((h // 8, w // 8, 8, 8), dtype=np.int32) if w % 8 == 0 and h % 8 == 0 else np.zeros(1, np.int32)
    _check(_load().rdct_ref_forward(_ptr(img, ctypes.c_uint8), pitch, w, h, _ptr(Y, ctypes.c_int32)), "forward")
    return Y


def forward_f64(img: np.ndarray, kind: int = KIND_RDCT) -> np.ndarray:
    """Orthonormal M A M^T per block in FP64 (M = C_orth or C); [nbh, nbw, 8, 8]."""
    img, pitch, w, h = _plane(img)
    Y = np.zeros((h // 8, w // 8, 8, 8))
    _check(_load().rdct_ref_forward_f64(_ptr(img, ctypes.c_uint8), pitch, w, h, kind, _ptr(Y, ctypes.c_double)),
           "forward_f64")
    return Y


def compress(Y: np.ndarray, r: int) -> np.ndarray:
    """First r zigzag coefficients of S Y S per block; [nblocks, r] FP64."""
    Yb = np.ascontiguousarray(Y, dtype=np.int32).reshape(-1, 64)
    out = np.zeros((Yb.shape[0], r))
    _check(_load().rdct_ref_compress(_ptr(Yb, ctypes.c_int32), Yb.shape[0], r, _ptr(out, ctypes.c_double)),
           "compress")
    return out


def inverse(Yc: np.ndarray, nbw: int, nbh: int, r: int, kind: int = KIND_RDCT) -> np.ndarray:
    """Reconstruct M^T Yhat M from packed zigzag coefficients; FP64 [8 nbh, 8 nbw]."""
    yc = np.ascontiguousarray(Yc, dtype=np.float64).reshape(-1)
    out = np.zeros((nbh * 8, nbw * 8))
    _check(_load().rdct_ref_inverse(_ptr(yc, ctypes.c_double), nbw, nbh, r, kind, _ptr(out, ctypes.c_double),
                                    nbw * 8), "inverse")
    return out


def fused(img: np.ndarray, r: int, kind: int = KIND_RDCT, want_xhat: bool = True, want_u8: bool = True,
          nthreads: int = 0):
    """Sec. 3 for one plane: returns (xhat or None, u8 or None, sse, sse_u8)."""
    img, pitch, w, h = _plane(img)
    xhat = np.zeros((h, w)) if want_xhat else None
    u8 = np.zeros((h, w), dtype=np.uint8) if want_u8 else None
    sse = np.zeros(1)
    sse_u8 = np.zeros(1)
    lib = _load()
    _check(lib.rdct_ref_fused(_ptr(img, ctypes.c_uint8), pitch, w, h, r, kind,
                              _ptr(xhat, ctypes.c_double) if xhat is not None else None,
                              _ptr(u8, ctypes.c_uint8) if u8 is not None else None,
                              _ptr(sse, ctypes.c_double), _ptr(sse_u8, ctypes.c_double), nthreads), "fused")
    return xhat, u8, float(sse[0]), float(sse_u8[0])


def sweep(img: np.ndarray, kind: int = KIND_RDCT, nthreads: int = 0) -> np.ndarray:
    """SSE for r = 1..64 by direct reconstruction at every r; FP64 [64]."""
    img, pitch, w, h = _plane(img)
    out = np.zeros(64)
    _check(_load().rdct_ref_sweep(_ptr(img, ctypes.c_uint8), pitch, w, h, kind, _ptr(out, ctypes.c_double),
                                  nthreads), "sweep")
    return out


def sse(ref: np.ndarray, rec: np.ndarray) -> float:
    """Sum of squared differences between a uint8 plane and a uint8 or float reconstruction."""
    ref, pitch, w, h = _plane(ref)
    out = np.zeros(1)
    lib = _load()
    if rec.dtype == np.uint8:
        rec = np.ascontiguousarray(rec)
        st = lib.rdct_ref_sse(_ptr(ref, ctypes.c_uint8), pitch, w, h, _ptr(rec, ctypes.c_uint8), None,
                              rec.shape[1], _ptr(out, ctypes.c_double))
    else:
        rec = np.ascontiguousarray(rec, dtype=np.float64)
        st = lib.rdct_ref_sse(_ptr(ref, ctypes.c_uint8), pitch, w, h, None, _ptr(rec, ctypes.c_double),
                              rec.shape[1], _ptr(out, ctypes.c_double))
    _check(st, "sse")
    return float(out[0])


def uqi(ref: np.ndarray, rec: np.ndarray, window: int = 8) -> float:
    """UQI (Wang & Bovik, cited in Sec. 3): mean over sliding window x window windows of
    [2 s_xy / (s_x^2 + s_y^2)] [2 mx my / (mx^2 + my^2)] (a factor with a zero denominator is 1)."""
    ref, pitch, w, h = _plane(ref)
    out = np.zeros(1)
    lib = _load()
    if rec.dtype == np.uint8:
        rec = np.ascontiguousarray(rec)
        st = lib.rdct_ref_uqi(_ptr(ref, ctypes.c_uint8), pitch, w, h, _ptr(rec, ctypes.c_uint8), None,
                              rec.shape[1], window, _ptr(out, ctypes.c_double))
    else:
        rec = np.ascontiguousarray(rec, dtype=np.float64)
        st = lib.rdct_ref_uqi(_ptr(ref, ctypes.c_uint8), pitch, w, h, None, _ptr(rec, ctypes.c_double),
                              rec.shape[1], window, _ptr(out, ctypes.c_double))
    _check(st, "uqi")
    return float(out[0])


def max_threads() -> int:
    return int(_load().rdct_ref_max_threads())


# ----------------------------------------------------------- quality measures

PEAK = 255.0  # 8-bit images (Sec. 3); the paper does not print the peak


def mse(sse_value: float, n_samples: int) -> float:
    """Sec. 3: mean squared error = SSE / number of samples."""
    return sse_value / n_samples


def psnr(mse_value: float) -> float:
    """Sec. 3: PSNR = 10 log10(255^2 / MSE); +inf when MSE = 0."""
    if mse_value == 0.0:
        return float("inf")
    return 10.0 * np.log10(PEAK * PEAK / mse_value)


def average(values) -> float:
    """Sec. 3: the average over images of a per-image figure (mean of the values)."""
    v = np.asarray(list(values), dtype=np.float64)
    return float(v.mean())


def ape(value: float, exact: float) -> float:
    """Sec. 3: absolute percentage error of a figure relative to the exact DCT's."""
    return 100.0 * abs(value - exact) / abs(exact)


# ------------------------------------------------------ spectral analysis (Sec. 2)

def transfer_function(T: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """H_m(w; T) = sum_n t_{m,n} exp(-j n w) for every row m; shape [8, len(omega)]."""
    n = np.arange(8)
    E = np.exp(-1j * np.outer(n, omega))  # [8 taps, n_omega]
    return np.asarray(T, dtype=np.float64) @ E


def spectral_error(T: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """D_m(w; T) = |H_m(w; C) - H_m(w; T)|^2; shape [8, len(omega)]."""
    return np.abs(transfer_function(dct_matrix(), omega) - transfer_function(T, omega)) ** 2


def error_energy(T: np.ndarray, n_points: int = 20001) -> np.ndarray:
    """eps_m(T) = integral over [0, pi] of D_m(w; T) dw (composite Simpson rule); shape [8]."""
    if n_points % 2 == 0:
        n_points += 1
    omega = np.linspace(0.0, np.pi, n_points)
    D = spectral_error(T, omega)
    hstep = omega[1] - omega[0]
    wts = np.ones(n_points)
    wts[1:-1:2] = 4.0
    wts[2:-1:2] = 2.0
    return (D @ wts) * hstep / 3.0
