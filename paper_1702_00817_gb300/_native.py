"""ctypes view of the C ABI in include/adct.h (argument marshalling only).

The functions exported here carry the C names (adct_create, adct_forward, ...)
with the C argument types.  Loading fails loudly when libadct.so has not been
built: there is no fallback implementation anywhere in the package.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

ADCT_OK = 0
ADCT_ERR_INVALID_ARG = 1
ADCT_ERR_SHAPE = 2
ADCT_ERR_ALIGN = 3
ADCT_ERR_OOM = 4
ADCT_ERR_CUDA = 5
ADCT_ERR_TIMEOUT = 6
ADCT_ERR_UNSUPPORTED = 7
ADCT_ERR_TOO_LARGE = 8
ADCT_ERR_CANCELLED = 9
NOALLOC_MAX_PLANES = 1024

ADCT_Q_NONE, ADCT_Q_STEP, ADCT_Q_ZONAL, ADCT_Q_STEP_ZONAL, ADCT_Q_ZONAL_ZZ = 0, 1, 2, 3, 4
ADCT_LAYOUT_PLANAR, ADCT_LAYOUT_INTERLEAVED = 0, 1

# Every symbol include/adct.h declares.
EXPORTS = (
    "adct_create", "adct_destroy", "adct_forward", "adct_quantise", "adct_inverse", "adct_roundtrip",
    "adct_forward_f32", "adct_backward_f32", "adct_set_launch", "adct_get_launch", "adct_roundtrip_graph",
    "adct_autotune", "adct_roundtrip_host", "adct_butterfly_host", "adct_kernel_timing", "adct_kernel_time",
    "adct_roundtrip_noalloc", "adct_quality", "adct_quality_dct", "adct_server_create", "adct_server_destroy", "adct_server_encode",
    "adct_server_decode", "adct_server_poll", "adct_server_stats", "adct_server_clock", "adct_shard_plan",
    "adct_checked_faults", "adct_server_cancel",
    "adct_status_string", "adct_last_error",
)


class adct_image(ctypes.Structure):
    _fields_ = [
        ("src", ctypes.c_void_p),
        ("dst", ctypes.c_void_p),
        ("coef", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("channels", ctypes.c_int32),
        ("layout", ctypes.c_int32),
        ("pitch", ctypes.c_int64),
        ("plane_stride", ctypes.c_int64),
    ]


class adct_quant(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("r", ctypes.c_int32), ("Q", ctypes.c_uint16 * 64)]


class adct_launch(ctypes.Structure):
    _fields_ = [
        ("threads_per_cta", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("stage_coef", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class adct_server_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("quant", adct_quant)]


class adct_completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("handle", ctypes.c_uint64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class adct_server_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("launches", "admitted", "evicted", "unknown_handle", "oversized",
                                              "errors", "store_entries", "arena_free_bytes")] + \
               [("max_overlap", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cancelled", ctypes.c_int64),
                ("latency_hist", ctypes.c_int64 * 32)]


class AdctError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libadct.so (built by __graft_entry__.build()).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _open(path or _build.LIB)
    return _lib


def load_checked() -> ctypes.CDLL:
    """Load libadct_checked.so, the build whose kernels check their own bounds
    (built by paper_1702_00817_gb300._build.build(checked=True)); a separate
    library instance next to the release one."""
    return _open(_build.LIB_CHECKED)


def _open(path: str) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    I = ctypes.POINTER(adct_image)
    Qp = ctypes.POINTER(adct_quant)
    L = ctypes.POINTER(adct_launch)
    sig = {
        "adct_create": ([ctypes.POINTER(ctypes.c_void_p), i32], i32),
        "adct_destroy": ([P], None),
        "adct_forward": ([P, I, i32, P], i32),
        "adct_quantise": ([P, I, i32, Qp, P], i32),
        "adct_inverse": ([P, I, i32, Qp, P], i32),
        "adct_roundtrip": ([P, I, i32, Qp, P], i32),
        "adct_forward_f32": ([P, P, P, i64, i32, i32, P, P], i32),
        "adct_backward_f32": ([P, P, P, P, i64, i32, i32, P, P], i32),
        "adct_set_launch": ([P, L], i32),
        "adct_get_launch": ([P, L], i32),
        "adct_roundtrip_graph": ([P, I, i32, Qp, P, ctypes.POINTER(i32)], i32),
        "adct_autotune": ([P, I, i32, Qp, P, i32, L, ctypes.POINTER(ctypes.c_float)], i32),
        "adct_roundtrip_host": ([P, I, i32, Qp, i64], i32),
        "adct_butterfly_host": ([P, i64, i32, ctypes.POINTER(i32)], i32),
        "adct_kernel_timing": ([P, i32], i32),
        "adct_kernel_time": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)], i32),
        "adct_roundtrip_noalloc": ([I, i32, Qp, P], i32),
        "adct_quality": ([P, I, i32, Qp, P, P], i32),
        "adct_quality_dct": ([P, I, i32, i32, P, P], i32),
        "adct_server_create": ([ctypes.POINTER(ctypes.c_void_p), i32, ctypes.POINTER(adct_server_config)], i32),
        "adct_server_destroy": ([P], None),
        "adct_server_encode": ([P, P, i32, i32, i64, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)], i32),
        "adct_server_decode": ([P, ctypes.c_uint64, P, i64, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "adct_server_poll": ([P, ctypes.POINTER(adct_completion), i32, i32], i32),
        "adct_server_stats": ([P, ctypes.POINTER(adct_server_stats_t)], i32),
        "adct_server_clock": ([], ctypes.c_double),
        "adct_shard_plan": ([I, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)], i32),
        "adct_checked_faults": ([P, ctypes.POINTER(ctypes.c_uint32)], i32),
        "adct_server_cancel": ([P, ctypes.c_uint64], i32),
        "adct_status_string": ([i32], ctypes.c_char_p),
        "adct_last_error": ([P], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def check(status: int, ctx=None, what: str = "", lib=None) -> None:
    """Raise AdctError for a non-OK status (lib: the library that owns ctx)."""
    if status != ADCT_OK:
        lib = lib if lib is not None else load()
        name = lib.adct_status_string(status).decode()
        msg = lib.adct_last_error(ctx).decode() if ctx else ""
        raise AdctError(status, f"{what}: {name} {msg}".strip())
