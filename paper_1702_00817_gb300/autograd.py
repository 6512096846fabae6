"""torch.autograd.Function over the float32 kernels (Sec. 2: C^ = D T orthogonal).

Forward: y = D T x T^T D per 8x8 block (plus the soft quantiser when Qsoft is
given), computed by adct_forward_f32.  Backward: the hand-written adjoint
kernel adct_backward_f32, gx = T^T D (gy * dz/dy) D T.  Only x is saved.
"""
from __future__ import annotations

import threading

import torch

from .codec import Codec

_codecs: dict[int, Codec] = {}
_lock = threading.Lock()


def default_codec(device: int) -> Codec:
    with _lock:
        c = _codecs.get(device)
        if c is None:
            c = _codecs[device] = Codec(device)
        return c


class ADCTFunction(torch.autograd.Function):
    """y = ADCTFunction.apply(x, Qsoft=None): x float32 [..., H, W] on a CUDA device."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, Qsoft=None):
        if not x.is_cuda:
            raise ValueError("ADCTFunction needs a CUDA tensor")
        xc = x.contiguous()
        codec = default_codec(xc.device.index or 0)
        y = codec.forward_f32(xc, Qsoft)
        ctx.save_for_backward(xc)
        ctx.Qsoft = Qsoft
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        (x,) = ctx.saved_tensors
        codec = default_codec(x.device.index or 0)
        gx = codec.backward_f32(x, gy.contiguous(), ctx.Qsoft)
        return gx, None
