"""Python binding of the codec's C ABI for torch tensors (marshalling only).

Every computation happens in libadct.so's CUDA kernels; this module turns
torch tensors into adct_image / adct_quant structures, passes the current
CUDA stream, and raises AdctError on a non-OK status.

Tensor conventions (matching include/adct.h):
  pixels  uint8 [C, H, W] or [H, W], unit stride along W (rows and planes may be pitched);
          with Image(..., interleaved=True) uint8 [H, W, C], C = 3 or 4, channels adjacent
  coef    int16, contiguous, block-major [C, Hb, Wb, 8, 8] with Hb = ceil(H/8), Wb = ceil(W/8)
          (ADCT_Q_ZONAL_ZZ: packed [C, Hb, Wb, r], zig-zag order)
  float   float32 [..., H, W] contiguous
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as N
from ._native import (ADCT_Q_NONE, ADCT_Q_STEP, ADCT_Q_STEP_ZONAL, ADCT_Q_ZONAL, ADCT_Q_ZONAL_ZZ,  # noqa: F401
                      AdctError)


def make_quant(mode: int, Q=None, r: int = 64) -> N.adct_quant:
    """Quantiser descriptor: mode ADCT_Q_*, Q an 8x8 step table (row-major), r kept zig-zag coefficients."""
    q = N.adct_quant()
    q.mode = int(mode)
    q.r = int(r)
    vals = [1] * 64 if Q is None else [int(v) for v in (Q.reshape(-1).tolist() if hasattr(Q, "reshape") else Q)]
    if len(vals) != 64:
        raise ValueError("Q needs 64 entries")
    for k, v in enumerate(vals):
        if not 0 <= v <= 65535:
            raise ValueError("Q entries must fit uint16")
        q.Q[k] = v
    return q


def coef_per_block(quant) -> int:
    """int16 coefficients stored per 8x8 block under `quant`: r for the packed zonal layout, else 64."""
    return int(quant.r) if quant is not None and quant.mode == ADCT_Q_ZONAL_ZZ and 0 <= quant.r <= 64 else 64


@dataclass
class Image:
    """One image for the codec: any of src/dst (uint8 pixels) and coef (int16);
    interleaved: the pixel tensors are [H, W, C] (HWC, C = 3 or 4)."""
    src: torch.Tensor | None = None
    dst: torch.Tensor | None = None
    coef: torch.Tensor | None = None
    interleaved: bool = False


def _pix_geometry(t: torch.Tensor, interleaved: bool = False):
    if t.dtype != torch.uint8:
        raise TypeError("pixel tensors must be uint8")
    if interleaved:
        if t.dim() != 3 or t.stride(2) != 1 or t.stride(1) != t.shape[2]:
            raise ValueError("interleaved pixel tensors are [H, W, C] with adjacent channels")
        H, W, C = t.shape
        # a single row's pitch is never used (torch may report any stride for it)
        return C, H, W, t.stride(0) if H > 1 else (W * C + 7) // 8 * 8, 0
    if t.dim() == 2:
        H, W = t.shape
        if t.stride(1) != 1 and W > 1:
            raise ValueError("pixel rows need unit stride")
        pitch = t.stride(0) if H > 1 else (W + 7) // 8 * 8
        return 1, H, W, pitch, pitch * H
    if t.dim() == 3:
        C, H, W = t.shape
        if t.stride(2) != 1 and W > 1:
            raise ValueError("pixel rows need unit stride")
        pitch = t.stride(1) if H > 1 else (W + 7) // 8 * 8
        return C, H, W, pitch, t.stride(0) if C > 1 else pitch * H
    raise ValueError("pixel tensors are [H, W] or [C, H, W]")


def _check_place(t: torch.Tensor, device, what: str):
    """device: None (no check), "cpu" (host tensors, the host pipeline) or a
    CUDA device index (device memory on that GPU)."""
    if device is None:
        return
    if device == "cpu":
        if t.is_cuda:
            raise ValueError(f"{what}: the host pipeline takes host tensors")
    elif not t.is_cuda or t.device.index != device:
        raise ValueError(f"{what} must be a CUDA tensor on cuda:{device}")


def image_struct(im, cpb: int = 64, device=None) -> N.adct_image:
    if isinstance(im, (tuple, list)):
        im = Image(*im)
    for t, what in ((im.src, "src"), (im.dst, "dst"), (im.coef, "coef")):
        if t is not None:
            _check_place(t, device, what)
    ref = im.src if im.src is not None else im.dst
    s = N.adct_image()
    if ref is not None:
        C, H, W, pitch, pstride = _pix_geometry(ref, im.interleaved)
        if im.src is not None and im.dst is not None:
            g2 = _pix_geometry(im.dst, im.interleaved)
            if g2 != (C, H, W, pitch, pstride):
                raise ValueError("src and dst must share shape, pitch and plane stride")
    elif im.coef is not None:
        # coefficient-only image: [C, Hb, Wb, 8, 8], or [C, Hb, Wb, r] packed
        if im.coef.dim() != (5 if cpb == 64 else 4):
            raise ValueError("a coefficient-only image needs coef shaped [C, Hb, Wb, 8, 8] "
                             "([C, Hb, Wb, r] for the packed zonal layout)")
        C, hb, wb = im.coef.shape[:3]
        H, W, pitch, pstride = hb * 8, wb * 8, wb * 8, hb * 8 * wb * 8
    else:
        raise ValueError("image has no tensors")
    if im.coef is not None:
        nb = ((H + 7) // 8) * ((W + 7) // 8)
        if im.coef.dtype != torch.int16 or not im.coef.is_contiguous() or im.coef.numel() != C * nb * cpb:
            raise ValueError(f"coef must be contiguous int16 with {cpb} elements per 8x8 block")
    s.src = im.src.data_ptr() if im.src is not None else None
    s.dst = im.dst.data_ptr() if im.dst is not None else None
    s.coef = im.coef.data_ptr() if im.coef is not None else None
    s.width, s.height, s.channels = W, H, C
    s.layout = N.ADCT_LAYOUT_INTERLEAVED if im.interleaved and ref is not None else N.ADCT_LAYOUT_PLANAR
    s.pitch, s.plane_stride = pitch, pstride
    return s


def image_array(images, quant=None, device=None):
    """adct_image array of `images`; device as in _check_place (the Codec
    passes its GPU, or "cpu" for the host pipeline)."""
    cpb = coef_per_block(quant)
    arr = (N.adct_image * max(1, len(images)))()
    for k, im in enumerate(images):
        arr[k] = image_struct(im, cpb, device)
    return arr


def _stream_handle(device: int, stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _f32(t: torch.Tensor, name: str, device: int | None = None, like: torch.Tensor | None = None):
    if t.dtype != torch.float32 or not t.is_contiguous() or t.dim() < 2:
        raise ValueError(f"{name} must be a contiguous float32 tensor [..., H, W]")
    _check_place(t, device, name)
    if like is not None and t.shape != like.shape:
        raise ValueError(f"{name} must have the shape of x")
    H, W = t.shape[-2], t.shape[-1]
    return t.numel() // (H * W), H, W


def _qsoft(Qsoft):
    if Qsoft is None:
        return None
    vals = [float(v) for v in (Qsoft.reshape(-1).tolist() if hasattr(Qsoft, "reshape") else Qsoft)]
    if len(vals) != 64:
        raise ValueError("Qsoft needs 64 entries")
    return (ctypes.c_float * 64)(*vals)


class Codec:
    """A library context bound to one CUDA device."""

    def __init__(self, device: int = 0, lib=None):
        self.lib = lib if lib is not None else N.load()
        self.device = int(device)
        h = ctypes.c_void_p()
        N.check(self.lib.adct_create(ctypes.byref(h), self.device), None, "adct_create", lib=self.lib)
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.adct_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- integer codec ------------------------------------------------------
    def _call(self, name, images, quant=None, stream=None):
        arr = image_array(images, quant, self.device)
        args = [self.ctx, arr, len(images)]
        if quant is not None:
            args.append(ctypes.byref(quant))
        args.append(_stream_handle(self.device, stream))
        N.check(getattr(self.lib, name)(*args), self.ctx, name, lib=self.lib)

    def forward(self, images, stream=None):
        self._call("adct_forward", images, None, stream)

    def quantise(self, images, quant, stream=None):
        self._call("adct_quantise", images, quant, stream)

    def inverse(self, images, quant, stream=None):
        self._call("adct_inverse", images, quant, stream)

    def roundtrip(self, images, quant, stream=None):
        self._call("adct_roundtrip", images, quant, stream)

    def roundtrip_graph(self, images, quant, stream=None) -> bool:
        arr = image_array(images, quant, self.device)
        rep = ctypes.c_int32(0)
        st = self.lib.adct_roundtrip_graph(self.ctx, arr, len(images), ctypes.byref(quant),
                                           _stream_handle(self.device, stream), ctypes.byref(rep))
        N.check(st, self.ctx, "adct_roundtrip_graph", lib=self.lib)
        return bool(rep.value)

    def set_launch(self, threads_per_cta=0, ctas_per_sm=0, stage_coef=-1):
        l = N.adct_launch(threads_per_cta, ctas_per_sm, stage_coef, 0)
        N.check(self.lib.adct_set_launch(self.ctx, ctypes.byref(l)), self.ctx, "adct_set_launch", lib=self.lib)

    def get_launch(self) -> dict:
        l = N.adct_launch()
        N.check(self.lib.adct_get_launch(self.ctx, ctypes.byref(l)), self.ctx, "adct_get_launch", lib=self.lib)
        return {f: getattr(l, f) for f, _ in N.adct_launch._fields_}

    def autotune(self, images, quant, reps: int = 5, stream=None, cache: str | None = None):
        """Pick the fastest launch shape for this batch (adct_autotune) and keep it
        in the context.  cache: a JSON file of earlier results keyed by the
        batch signature (device, image shapes and layouts, which outputs,
        quantiser); a hit applies the stored shape without measuring.  Returns
        (shape, mean microseconds; None on a cache hit)."""
        key = self._signature(images, quant) if cache else None
        if cache:
            import json
            import os
            table = json.load(open(cache)) if os.path.exists(cache) else {}
            if key in table:
                shape = table[key]["launch"]
                self.set_launch(shape["threads_per_cta"], shape["ctas_per_sm"] or -1, shape["stage_coef"])
                return shape, None
        arr = image_array(images, quant, self.device)
        best = N.adct_launch()
        us = ctypes.c_float(0)
        st = self.lib.adct_autotune(self.ctx, arr, len(images), ctypes.byref(quant),
                                    _stream_handle(self.device, stream), int(reps), ctypes.byref(best),
                                    ctypes.byref(us))
        N.check(st, self.ctx, "adct_autotune", lib=self.lib)
        shape = {f: getattr(best, f) for f, _ in N.adct_launch._fields_}
        if cache:
            table = json.load(open(cache)) if os.path.exists(cache) else {}
            table[key] = {"launch": shape, "us": us.value}
            tmp = f"{cache}.{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return shape, us.value

    def _signature(self, images, quant) -> str:
        import hashlib
        parts = [torch.cuda.get_device_name(self.device), f"mode={quant.mode} r={quant.r}"]
        for im in images:
            im = Image(*im) if isinstance(im, (tuple, list)) else im
            s = image_struct(im, coef_per_block(quant))
            parts.append(f"{s.width}x{s.height}x{s.channels}/{s.layout}/{int(bool(s.coef))}{int(bool(s.dst))}")
        return hashlib.sha256("|".join(parts).encode()).hexdigest()[:24]

    def roundtrip_host(self, images, quant, chunk_bytes: int = 32 << 20):
        """End-to-end round trip on host (ideally pinned) tensors; synchronous."""
        arr = image_array(images, quant, "cpu")
        st = self.lib.adct_roundtrip_host(self.ctx, arr, len(images), ctypes.byref(quant), int(chunk_bytes))
        N.check(st, self.ctx, "adct_roundtrip_host", lib=self.lib)

    def quality(self, images, quant, stream=None) -> torch.Tensor:
        """Per-plane sum of squared round-trip error (int64 tensor on the device)."""
        arr = image_array(images, None, self.device)
        planes = sum(image_struct(im).channels for im in images)
        sse = torch.empty(max(1, planes), dtype=torch.int64, device=torch.device("cuda", self.device))
        st = self.lib.adct_quality(self.ctx, arr, len(images), ctypes.byref(quant), sse.data_ptr(),
                                   _stream_handle(self.device, stream))
        N.check(st, self.ctx, "adct_quality", lib=self.lib)
        return sse[:planes]

    def quality_dct(self, images, r: int, stream=None) -> torch.Tensor:
        """Per-plane sum of squared error of the exact-DCT zonal round trip keeping r coefficients."""
        arr = image_array(images, None, self.device)
        planes = sum(image_struct(im).channels for im in images)
        sse = torch.empty(max(1, planes), dtype=torch.int64, device=torch.device("cuda", self.device))
        st = self.lib.adct_quality_dct(self.ctx, arr, len(images), int(r), sse.data_ptr(),
                                       _stream_handle(self.device, stream))
        N.check(st, self.ctx, "adct_quality_dct", lib=self.lib)
        return sse[:planes]

    def checked_faults(self) -> int:
        """Bounds-check fault bits of a checked-build context (waits for the
        device, then clears them); AdctError(UNSUPPORTED) on the release build."""
        w = ctypes.c_uint32(0)
        N.check(self.lib.adct_checked_faults(self.ctx, ctypes.byref(w)), self.ctx, "adct_checked_faults",
                lib=self.lib)
        return w.value

    def kernel_timing(self, enable: bool):
        N.check(self.lib.adct_kernel_timing(self.ctx, 1 if enable else 0), self.ctx, "adct_kernel_timing",
                lib=self.lib)

    def kernel_time(self):
        """(summed kernel ms, kernels launched) since the previous query."""
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        N.check(self.lib.adct_kernel_time(self.ctx, ctypes.byref(ms), ctypes.byref(n)), self.ctx, "adct_kernel_time",
                lib=self.lib)
        return ms.value, n.value

    # -- float variant ------------------------------------------------------
    def forward_f32(self, x: torch.Tensor, Qsoft=None, out: torch.Tensor | None = None, stream=None):
        planes, H, W = _f32(x, "x", self.device)
        y = torch.empty_like(x) if out is None else out
        _f32(y, "out", self.device, x)
        st = self.lib.adct_forward_f32(self.ctx, x.data_ptr(), y.data_ptr(), planes, H, W, _qsoft(Qsoft),
                                       _stream_handle(self.device, stream))
        N.check(st, self.ctx, "adct_forward_f32", lib=self.lib)
        return y

    def backward_f32(self, x: torch.Tensor, gy: torch.Tensor, Qsoft=None, out: torch.Tensor | None = None,
                     stream=None):
        planes, H, W = _f32(x, "x", self.device)
        _f32(gy, "gy", self.device, x)
        gx = torch.empty_like(x) if out is None else out
        _f32(gx, "out", self.device, x)
        st = self.lib.adct_backward_f32(self.ctx, x.data_ptr(), gy.data_ptr(), gx.data_ptr(), planes, H, W,
                                        _qsoft(Qsoft), _stream_handle(self.device, stream))
        N.check(st, self.ctx, "adct_backward_f32", lib=self.lib)
        return gx


def shard_plan(shapes, world: int, rank: int):
    """Indices of the images of `rank` in the balanced no-collective partition
    of a batch over `world` GPUs (adct_shard_plan), and the largest per-rank
    block total.  shapes: (height, width) or (channels, height, width) tuples."""
    n = len(shapes)
    arr = (N.adct_image * max(1, n))()
    for k, sh in enumerate(shapes):
        c, h, w = (1, *sh) if len(sh) == 2 else sh
        arr[k].width, arr[k].height, arr[k].channels = int(w), int(h), int(c)
        arr[k].pitch, arr[k].plane_stride = int(w), int(w) * int(h)
    out = (ctypes.c_int32 * max(1, n))()
    count = ctypes.c_int32(0)
    mx = ctypes.c_int64(0)
    lib = N.load()
    N.check(lib.adct_shard_plan(arr, n, int(world), int(rank), out, ctypes.byref(count), ctypes.byref(mx)), None,
            "adct_shard_plan")
    return [out[k] for k in range(count.value)], mx.value


def butterfly_host(vectors, inverse: bool = False):
    """Run the library's 8-point butterfly on the host; returns (outputs, adds per transform)."""
    import numpy as np
    v = np.ascontiguousarray(np.asarray(vectors, dtype=np.int32).reshape(-1, 8)).copy()
    adds = ctypes.c_int32(0)
    lib = N.load()
    st = lib.adct_butterfly_host(v.ctypes.data, v.shape[0], 1 if inverse else 0, ctypes.byref(adds))
    N.check(st, None, "adct_butterfly_host")
    return v, adds.value
