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
