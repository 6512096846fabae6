"""The round trip that allocates nothing, checked against the ordinary one.

adct_roundtrip_noalloc serves callers that cannot call cudaMalloc (a plug-in
bound to its host application's device-memory pool or budget, a latency-critical
loop that cannot take cudaMalloc's implicit device synchronisation, a service
that must not run out of memory after start-up).  It keeps its per-call
descriptor table in a fixed device array inside the library instead of a
context workspace.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a
fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1702_00817_gb300 import _native, inputs
from paper_1702_00817_gb300.codec import ADCT_Q_STEP, ADCT_Q_ZONAL, Codec, Image, image_array, make_quant

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return _native.load()


def _batch(seed):
    sizes = inputs.ragged_sizes(7, seed=seed, lo_log2=4.0, hi_log2=9.0)
    return inputs.ragged_batch(sizes, channels=2, base_seed=seed)


def _tensors(imgs, with_coef=True, with_dst=True):
    srcs = [torch.from_numpy(x).to(DEV) for x in imgs]
    dsts = [torch.full_like(s, 3) if with_dst else None for s in srcs]
    coefs = [torch.full((x.shape[0], x.shape[1] // 8, x.shape[2] // 8, 8, 8), 77, dtype=torch.int16, device=DEV)
             if with_coef else None for x in imgs]
    return [Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)]


def test_noalloc_matches_roundtrip_on_two_calls_in_a_row(lib):
    codec = Codec(0)
    stream = torch.cuda.current_stream(DEV)
    sh = ctypes.c_void_p(stream.cuda_stream)
    quants = [make_quant(ADCT_Q_STEP, inputs.step_table(4)), make_quant(ADCT_Q_ZONAL, None, 10)]
    for call, q in enumerate(quants):
        imgs = _batch(900 + call)
        ref = _tensors(imgs)
        new = _tensors(imgs)
        codec.roundtrip(ref, q)
        st = lib.adct_roundtrip_noalloc(image_array(new), len(new), ctypes.byref(q), sh)
        assert st == _native.ADCT_OK, lib.adct_status_string(st)
        torch.cuda.synchronize()
        for a, b in zip(ref, new):
            assert torch.equal(a.dst, b.dst)   # integer path: exact agreement
            assert torch.equal(a.coef, b.coef)
    codec.close()


def test_noalloc_rejects_batches_beyond_its_table(lib):
    n = _native.NOALLOC_MAX_PLANES + 1
    px = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    out = torch.zeros_like(px)
    arr = image_array([Image(px, out, None)] * n)
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    sh = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    assert lib.adct_roundtrip_noalloc(arr, n, ctypes.byref(q), sh) == _native.ADCT_ERR_TOO_LARGE
    # exactly the maximum is accepted
    assert lib.adct_roundtrip_noalloc(arr, n - 1, ctypes.byref(q), sh) == _native.ADCT_OK
    torch.cuda.synchronize()
    expect = np.full((8, 8), 0, np.uint8)
    assert np.array_equal(out.cpu().numpy(), expect)  # an all-zero block reconstructs to zero at this step table


def _pitched(shape, interleaved, fill=0):
    """A uint8 image with rows padded to a multiple of 8 bytes ([C, H, W], or
    [H, W, C] interleaved), as the codec's 8-byte row alignment requires."""
    if interleaved:
        H, W, C = shape
        pitch = (W * C + 15) // 16 * 16
        buf = torch.full((H, pitch), fill, dtype=torch.uint8, device=DEV)
        return buf.as_strided((H, W, C), (pitch, C, 1))
    C, H, W = shape
    pitch = (W + 15) // 16 * 16
    buf = torch.full((C, H, pitch), fill, dtype=torch.uint8, device=DEV)
    return buf[:, :, :W]


# (channels, height, width, interleaved): planar with and without edge blocks,
# 3- and 4-channel interleaved with and without them -- every layout class
# of the call, so the per-class tables sit back to back in the fixed array
MIXED = [(1, 45, 83, False), (2, 64, 72, False), (3, 37, 50, True), (4, 48, 64, True),
         (3, 40, 56, True), (1, 21, 19, False), (4, 13, 29, True)]


def _mixed_images(seed, q):
    from paper_1702_00817_gb300.codec import coef_per_block
    cpb = coef_per_block(q)
    out = []
    for k, (C, H, W, inter) in enumerate(MIXED):
        x = inputs.synth_image(H, W, seed + k, channels=C)  # [C, H, W]
        src = _pitched((H, W, C) if inter else (C, H, W), inter)
        src.copy_(torch.from_numpy(np.moveaxis(x, 0, -1).copy() if inter else x).to(DEV))
        dst = _pitched(src.shape, inter, fill=5)
        hb, wb = (H + 7) // 8, (W + 7) // 8
        coef = torch.full((C, hb, wb, 8, 8) if cpb == 64 else (C, hb, wb, cpb), 99, dtype=torch.int16, device=DEV)
        out.append(Image(src, dst, coef, inter))
    return out


def test_noalloc_mixed_layouts_and_packed_zonal_match_roundtrip(lib):
    from paper_1702_00817_gb300.codec import ADCT_Q_ZONAL_ZZ
    codec = Codec(0)
    sh = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    quants = [make_quant(ADCT_Q_ZONAL_ZZ, None, 10), make_quant(ADCT_Q_STEP, inputs.step_table(1)),
              make_quant(ADCT_Q_ZONAL_ZZ, None, 7), make_quant(ADCT_Q_STEP, inputs.step_table(4))]
    for call, q in enumerate(quants):  # consecutive calls: each rewrites the fixed table
        ref = _mixed_images(700 + 10 * call, q)
        new = _mixed_images(700 + 10 * call, q)
        codec.roundtrip(ref, q)
        st = lib.adct_roundtrip_noalloc(image_array(new, q), len(new), ctypes.byref(q), sh)
        assert st == _native.ADCT_OK, lib.adct_status_string(st)
        torch.cuda.synchronize()
        for a, b in zip(ref, new):
            assert torch.equal(a.dst, b.dst)
            assert torch.equal(a.coef, b.coef)
    codec.close()


def test_noalloc_from_a_thread_with_a_small_stack(lib):
    # Host applications may call from threads with small stacks; the 72 KiB
    # table is not on the stack.  The thread gets the smallest stack the
    # platform accepts: 64 KiB, or 128 KiB where that is the minimum (aarch64
    # with 64 KiB pages).
    import threading
    codec = Codec(0)
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    ref, new = _mixed_images(800, q), _mixed_images(800, q)
    codec.roundtrip(ref, q)
    torch.cuda.synchronize()
    arr = image_array(new, q)
    stream = torch.cuda.current_stream(DEV)
    out = []

    def call():  # device 0 is the runtime's default on a new thread
        out.append(lib.adct_roundtrip_noalloc(arr, len(new), ctypes.byref(q), ctypes.c_void_p(stream.cuda_stream)))

    old = None
    for size in (65536, 131072):
        try:
            old = threading.stack_size(size)
            break
        except ValueError:
            continue
    assert old is not None
    try:
        t = threading.Thread(target=call)
        t.start()
        t.join()
    finally:
        threading.stack_size(old)
    assert out == [_native.ADCT_OK]
    torch.cuda.synchronize()
    for a, b in zip(ref, new):
        assert torch.equal(a.dst, b.dst)
        assert torch.equal(a.coef, b.coef)
    codec.close()
