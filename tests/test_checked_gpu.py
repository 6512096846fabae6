"""The checked build (libadct_checked.so: kernels that verify every tile
position lies inside its plane's blocks and no pixel copy passes the end of a
row, reporting violations in a fault word instead of touching memory) runs
every layout, quantiser mode and kind with no fault and with outputs equal to
the release build's, bit for bit.  A stand-in for a memory checker, which is
not available on this machine."""
import numpy as np
import pytest
import torch

from paper_1702_00817_gb300 import _build, _native, inputs
from paper_1702_00817_gb300.codec import (ADCT_Q_STEP, ADCT_Q_ZONAL, ADCT_Q_ZONAL_ZZ, AdctError, Codec, Image,
                                          make_quant)

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def pair():
    import __graft_entry__
    __graft_entry__.build()
    _build.build(checked=True)
    release, checked = Codec(0), Codec(0, lib=_native.load_checked())
    yield release, checked
    release.close()
    checked.close()


def _pitched(x, interleaved):
    if interleaved:
        H, W, C = x.shape
        pitch = (W * C + 7) // 8 * 8
        buf = torch.zeros((H, pitch), dtype=torch.uint8, device=DEV)
        v = buf[:, :W * C].view(H, W, C)
    else:
        C, H, W = x.shape
        pitch = (W + 7) // 8 * 8
        buf = torch.zeros((C, H, pitch), dtype=torch.uint8, device=DEV)
        v = buf[:, :, :W]
    v.copy_(torch.from_numpy(np.ascontiguousarray(x)))
    return v


def _batch():
    out = []
    for k, (h, w) in enumerate(inputs.ragged_sizes(10, seed=44, lo_log2=3.0, hi_log2=9.0)):
        out.append((inputs.synth_image(h, w, 60 + k, channels=1 + k % 3), False))
    for k, (h, w) in enumerate([(45, 83), (8, 8), (130, 250), (17, 9)]):
        out.append((inputs.synth_image(h, w, 70 + k, channels=1 + k % 2), False))  # edge blocks
        x = np.moveaxis(inputs.synth_image(h, w, 80 + k, channels=3 + k % 2), 0, -1).copy()
        out.append((x, True))
    return out


@pytest.mark.parametrize("mode,s,r", [(ADCT_Q_STEP, 4, 64), (ADCT_Q_STEP, 1, 64), (ADCT_Q_ZONAL, None, 10),
                                      (ADCT_Q_ZONAL_ZZ, None, 10), (ADCT_Q_ZONAL_ZZ, None, 3)])
def test_checked_build_runs_clean_and_equal(pair, mode, s, r):
    release, checked = pair
    q = make_quant(mode, inputs.step_table(s) if s else None, r)
    imgs = _batch()
    results = []
    for codec in (release, checked):
        srcs = [_pitched(x, inter) for x, inter in imgs]
        dsts = [_pitched(np.zeros_like(x), inter) for x, inter in imgs]
        coefs = []
        for x, inter in imgs:
            C = x.shape[2] if inter else x.shape[0]
            H, W = (x.shape[0], x.shape[1]) if inter else (x.shape[1], x.shape[2])
            tail = (r,) if mode == ADCT_Q_ZONAL_ZZ else (8, 8)
            coefs.append(torch.zeros((C, (H + 7) // 8, (W + 7) // 8) + tail, dtype=torch.int16, device=DEV))
        ims = [Image(a, b, c, inter) for a, b, c, (_, inter) in zip(srcs, dsts, coefs, imgs)]
        codec.roundtrip(ims, q)  # full round trip
        codec.roundtrip([Image(a, b, None, inter) for a, b, (_, inter) in zip(srcs, dsts, imgs)], q)  # pixels only
        inv = [_pitched(np.zeros_like(x), inter) for x, inter in imgs]
        codec.inverse([Image(None, o, c, inter) for o, c, (_, inter) in zip(inv, coefs, imgs)], q)
        sse = codec.quality([Image(a, None, None, inter) for a, (_, inter) in zip(srcs, imgs)], q)
        torch.cuda.synchronize()
        results.append(([d.cpu() for d in dsts], [c.cpu() for c in coefs], [o.cpu() for o in inv], sse.cpu()))
    assert checked.checked_faults() == 0
    for a, b in zip(results[0][0] + results[0][1] + results[0][2], results[1][0] + results[1][1] + results[1][2]):
        assert torch.equal(a, b)
    assert torch.equal(results[0][3], results[1][3])


def test_release_build_reports_no_checks(pair):
    release, _ = pair
    with pytest.raises(AdctError) as e:
        release.checked_faults()
    assert e.value.status == _native.ADCT_ERR_UNSUPPORTED
