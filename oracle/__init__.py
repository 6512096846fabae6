"""Oracle for the 14-addition approximate DCT codec (Bayer & Cintra, 1702.00817).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark are the only callers.  The product library never imports this
package, and this package never imports the product.  The arithmetic lives in
``adct_oracle.c`` (plain dense-matrix C, int64 and double); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Sections cited: Sec. 2 (matrix T, D, D^2 merged into quantisation,
orthogonality), Sec. 3 (8x8 blockwise 2D transform, zig-zag zonal retention,
inverse procedure).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adct_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_NONE, MODE_STEP, MODE_ZONAL, MODE_STEP_ZONAL = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile adct_oracle.c into liboracle.so with gcc (host architecture)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.oracle_matrix_T.argtypes = [P]
            lib.oracle_scale_exponents.argtypes = [P]
            lib.oracle_zigzag_rank.argtypes = [P]
            lib.oracle_forward.argtypes = [P, i64, i32, i32, P]
            lib.oracle_quantise.argtypes = [P, i64, i32, P, i32, P]
            lib.oracle_inverse.argtypes = [P, i32, P, P, i64, i32, i32]
            lib.oracle_roundtrip.argtypes = [P, i64, P, i64, i32, i32, i32, P, i32, P, P]
            lib.oracle_forward_f64.argtypes = [P, i64, i32, i32, P, P, P]
            lib.oracle_backward_f64.argtypes = [P, P, i64, i32, i32, P, P]
            lib.oracle_dct_matrix.argtypes = [P]
            lib.oracle_dct_zonal.argtypes = [P, i64, i32, i32, i32, P, i64]
            for f in ("oracle_forward", "oracle_quantise", "oracle_inverse", "oracle_roundtrip",
                      "oracle_forward_f64", "oracle_backward_f64", "oracle_dct_zonal"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _plane(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x)
    if x.dtype != np.uint8 or x.ndim != 2:
        raise ValueError("expected a 2-D uint8 plane")
    return x


def matrix_T() -> np.ndarray:
    out = np.zeros(64, np.int64)
    _load().oracle_matrix_T(_p(out))
    return out.reshape(8, 8)


def scale_exponents() -> np.ndarray:
    out = np.zeros(8, np.int32)
    _load().oracle_scale_exponents(_p(out))
    return out


def zigzag_rank() -> np.ndarray:
    out = np.zeros(64, np.int32)
    _load().oracle_zigzag_rank(_p(out))
    return out.reshape(8, 8)


def _qtable(Q) -> np.ndarray:
    if Q is None:
        return np.ones(64, np.uint16)
    q = np.ascontiguousarray(np.asarray(Q, dtype=np.uint16).reshape(64))
    return q


def forward(plane: np.ndarray) -> np.ndarray:
    """Z = T (X - 128) T^T per 8x8 block; int64 block-major [H/8, W/8, 8, 8]."""
    x = np.ascontiguousarray(_plane(plane))
    H, W = x.shape
    Z = np.zeros((H // 8, W // 8, 8, 8), np.int64)
    if _load().oracle_forward(_p(x), W, W, H, _p(Z)) != 0:
        raise ValueError("oracle_forward: bad shape")
    return Z


def quantise(Z: np.ndarray, mode: int, Q=None, r: int = 64) -> np.ndarray:
    Zc = np.ascontiguousarray(Z, dtype=np.int64)
    q = np.zeros_like(Zc)
    Qt = _qtable(Q)
    if _load().oracle_quantise(_p(Zc), Zc.size // 64, int(mode), _p(Qt), int(r), _p(q)) != 0:
        raise ValueError("oracle_quantise: bad parameters")
    return q


def inverse(q: np.ndarray, mode: int, Q=None) -> np.ndarray:
    """Dequantise (D^2 merged) and invert block-major q [H/8, W/8, 8, 8] into a uint8 plane."""
    qc = np.ascontiguousarray(q, dtype=np.int64)
    hb, wb = qc.shape[0], qc.shape[1]
    dst = np.zeros((hb * 8, wb * 8), np.uint8)
    Qt = _qtable(Q)
    if _load().oracle_inverse(_p(qc), int(mode), _p(Qt), _p(dst), wb * 8, wb * 8, hb * 8) != 0:
        raise ValueError("oracle_inverse: bad parameters")
    return dst


def roundtrip(plane: np.ndarray, mode: int, Q=None, r: int = 64):
    """Returns (q int64 block-major, reconstructed uint8 plane)."""
    x = np.ascontiguousarray(_plane(plane))
    H, W = x.shape
    nb = (H // 8) * (W // 8)
    scratch = np.empty(2 * nb * 64, np.int64)
    q = np.zeros((H // 8, W // 8, 8, 8), np.int64)
    dst = np.zeros_like(x)
    Qt = _qtable(Q)
    rc = _load().oracle_roundtrip(_p(x), W, _p(dst), W, W, H, int(mode), _p(Qt), int(r),
                                  _p(scratch), _p(q))
    if rc != 0:
        raise ValueError("oracle_roundtrip: bad parameters")
    return q, dst


def roundtrip_pixels_only(plane: np.ndarray, mode: int, Q, r: int, scratch: np.ndarray,
                          dst: np.ndarray) -> None:
    """Round trip writing only the reconstructed plane (used for CPU timing)."""
    H, W = plane.shape
    Qt = _qtable(Q)
    rc = _load().oracle_roundtrip(_p(plane), W, _p(dst), W, W, H, int(mode), _p(Qt), int(r),
                                  _p(scratch), None)
    if rc != 0:
        raise ValueError("oracle_roundtrip: bad parameters")


def forward_f64(x: np.ndarray, Qsoft=None, want_y: bool = False):
    """Float variant: y = D T x T^T D per block, z = y - (Q/2pi) sin(2pi y/Q).

    x: [planes, H, W] (any float dtype, computed in float64)."""
    xc = np.ascontiguousarray(x, dtype=np.float64)
    planes = int(np.prod(xc.shape[:-2])) if xc.ndim > 2 else 1
    H, W = xc.shape[-2], xc.shape[-1]
    z = np.zeros_like(xc)
    y = np.zeros_like(xc) if want_y else None
    Qs = None if Qsoft is None else np.ascontiguousarray(np.asarray(Qsoft, np.float64).reshape(64))
    if _load().oracle_forward_f64(_p(xc), planes, H, W, _p(Qs), _p(y), _p(z)) != 0:
        raise ValueError("oracle_forward_f64: bad shape")
    return (z, y) if want_y else z


def backward_f64(x: np.ndarray, gz: np.ndarray, Qsoft=None) -> np.ndarray:
    xc = np.ascontiguousarray(x, dtype=np.float64)
    gc = np.ascontiguousarray(gz, dtype=np.float64)
    planes = int(np.prod(xc.shape[:-2])) if xc.ndim > 2 else 1
    H, W = xc.shape[-2], xc.shape[-1]
    gx = np.zeros_like(xc)
    Qs = None if Qsoft is None else np.ascontiguousarray(np.asarray(Qsoft, np.float64).reshape(64))
    if _load().oracle_backward_f64(_p(xc), _p(gc), planes, H, W, _p(Qs), _p(gx)) != 0:
        raise ValueError("oracle_backward_f64: bad shape")
    return gx


def dct_matrix() -> np.ndarray:
    out = np.zeros(64, np.float64)
    _load().oracle_dct_matrix(_p(out))
    return out.reshape(8, 8)


def dct_zonal(plane: np.ndarray, r: int) -> np.ndarray:
    """Exact-DCT zonal round trip of a uint8 plane keeping r zig-zag coefficients (Sec. 3 comparator)."""
    x = np.ascontiguousarray(_plane(plane))
    H, W = x.shape
    dst = np.zeros_like(x)
    if _load().oracle_dct_zonal(_p(x), W, W, H, int(r), _p(dst), W) != 0:
        raise ValueError("oracle_dct_zonal: bad parameters")
    return dst


def sse(a: np.ndarray, b: np.ndarray) -> int:
    """Sum of squared differences of two uint8 planes (exact)."""
    d = a.astype(np.int64) - b.astype(np.int64)
    return int((d * d).sum())
