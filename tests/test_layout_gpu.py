"""Edge extension (sides not multiples of 8) and channel-interleaved (HWC)
images against the oracle, bit for bit.

The oracle works on planar planes whose sides are multiples of 8; a test
extends each plane by replicating its last column and row (numpy edge
padding, the JPEG convention the library implements) and splits interleaved
images into planes.  Reconstructions are compared on the image's own pixels,
and the bytes beyond them (row padding, guard rows) must stay untouched."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import _native, inputs
from paper_1702_00817_gb300.codec import (ADCT_Q_NONE, ADCT_Q_STEP, ADCT_Q_ZONAL, ADCT_Q_ZONAL_ZZ, AdctError, Codec,
                                          Image, image_array, make_quant)

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
MODES = {ADCT_Q_NONE: oracle.MODE_NONE, ADCT_Q_STEP: oracle.MODE_STEP, ADCT_Q_ZONAL: oracle.MODE_ZONAL,
         ADCT_Q_ZONAL_ZZ: oracle.MODE_ZONAL}
ORDER = np.argsort(oracle.zigzag_rank().reshape(64))
GUARD = 0xA5
QUANTS = [(ADCT_Q_STEP, 4, 64), (ADCT_Q_STEP, 1, 64), (ADCT_Q_ZONAL, None, 10), (ADCT_Q_ZONAL_ZZ, None, 10),
          (ADCT_Q_NONE, None, 64)]


@pytest.fixture(scope="module")
def codec():
    import __graft_entry__
    __graft_entry__.build()
    c = Codec(0)
    yield c
    c.close()


def _quant(mode, s, r):
    return make_quant(mode, inputs.step_table(s) if s else None, r)


def _ref(plane, mode, s, r):
    """Oracle (q as stored for this mode, reconstruction) for one planar plane of any size."""
    H, W = plane.shape
    padded = np.pad(plane, ((0, (-H) % 8), (0, (-W) % 8)), mode="edge")
    q, rec = oracle.roundtrip(padded, MODES[mode], inputs.step_table(s) if s else None, r)
    if mode == ADCT_Q_ZONAL_ZZ:
        q = q.reshape(q.shape[0], q.shape[1], 64)[:, :, ORDER[:r]]
    return q, rec[:H, :W]


def _coef(C, H, W, mode, r):
    tail = (r,) if mode == ADCT_Q_ZONAL_ZZ else (8, 8)
    return torch.full((C, (H + 7) // 8, (W + 7) // 8) + tail, 77, dtype=torch.int16, device=DEV)


def _pitched(x: np.ndarray, interleaved: bool):
    """Device copy of a planar [C, H, W] or interleaved [H, W, C] image in a
    buffer whose rows are a multiple of 8 bytes plus 8 guard bytes, with a
    guard row below; returns (view, whole buffer)."""
    if interleaved:
        H, W, C = x.shape
        rowb = W * C
    else:
        C, H, W = x.shape
        rowb = W
    pitch = (rowb + 7) // 8 * 8 + 8
    if interleaved:
        buf = torch.full((H + 1, pitch), GUARD, dtype=torch.uint8, device=DEV)
        view = buf[:H, :rowb].view(H, W, C)
    else:
        buf = torch.full((C, H + 1, pitch), GUARD, dtype=torch.uint8, device=DEV)
        view = buf[:, :H, :W]
    view.copy_(torch.from_numpy(np.ascontiguousarray(x)))
    return view, buf


def _planes(x, interleaved):
    return [x[:, :, c] for c in range(x.shape[2])] if interleaved else [x[c] for c in range(x.shape[0])]


def _check(codec, imgs, mode, s, r, with_coef=True, with_dst=True):
    """One call over imgs = [(array, interleaved)]; compare every plane with the oracle."""
    q = _quant(mode, s, r)
    srcs, dsts, coefs, bufs = [], [], [], []
    for x, inter in imgs:
        src, _ = _pitched(x, inter)
        dst, dbuf = _pitched(np.zeros_like(x), inter) if with_dst else (None, None)
        if with_dst:
            dbuf.fill_(GUARD)
        C = x.shape[2] if inter else x.shape[0]
        H, W = (x.shape[0], x.shape[1]) if inter else (x.shape[1], x.shape[2])
        srcs.append(src)
        dsts.append(dst)
        bufs.append(dbuf)
        coefs.append(_coef(C, H, W, mode, r) if with_coef else None)
    codec.roundtrip([Image(s_, d_, c_, inter) for s_, d_, c_, (_, inter) in zip(srcs, dsts, coefs, imgs)], q)
    sse = codec.quality([Image(s_, None, None, inter) for s_, (_, inter) in zip(srcs, imgs)], q).cpu().numpy()
    torch.cuda.synchronize()
    pid = 0
    for (x, inter), d, c, b in zip(imgs, dsts, coefs, bufs):
        for k, plane in enumerate(_planes(x, inter)):
            qref, rec = _ref(np.ascontiguousarray(plane), mode, s, r)
            if with_coef:
                assert np.array_equal(c[k].cpu().numpy().astype(np.int64), qref), (x.shape, inter, k)
            if with_dst:
                out = d[:, :, k] if inter else d[k]
                assert np.array_equal(out.cpu().numpy(), rec), (x.shape, inter, k)
            assert int(sse[pid]) == oracle.sse(rec, np.ascontiguousarray(plane)), (x.shape, inter, k)
            pid += 1
        if with_dst:  # nothing written outside the image
            H = x.shape[0] if inter else x.shape[1]
            rowb = x.shape[1] * x.shape[2] if inter else x.shape[2]
            bb = b.cpu().numpy()
            if inter:
                assert (bb[:H, rowb:] == GUARD).all() and (bb[H:] == GUARD).all()
            else:
                assert (bb[:, :H, rowb:] == GUARD).all() and (bb[:, H:] == GUARD).all()
    return coefs


# (100, 61), (37, 250), (75, 93): interior and both edge strips in separate launches;
# (72, 93): right strip only; (75, 96): bottom strip only; the small ones stay whole
EDGE_SIZES = [(1, 1), (7, 13), (9, 17), (15, 8), (8, 15), (100, 61), (37, 250), (64, 64), (75, 93), (72, 93),
              (75, 96)]


@pytest.mark.parametrize("mode,s,r", QUANTS)
def test_edge_extension_planar(codec, mode, s, r):
    imgs = [(inputs.synth_image(h, w, 10 + k, channels=1 + k % 2), False) for k, (h, w) in enumerate(EDGE_SIZES)]
    _check(codec, imgs, mode, s, r)


@pytest.mark.parametrize("channels", [3, 4])
@pytest.mark.parametrize("mode,s,r", QUANTS)
def test_interleaved(codec, channels, mode, s, r):
    sizes = [(8, 8), (24, 40), (27, 45), (120, 256), (1, 9), (73, 31), (75, 93), (72, 93), (75, 96)]
    imgs = [(np.moveaxis(inputs.synth_image(h, w, 40 + k, channels=channels), 0, -1).copy(), True)
            for k, (h, w) in enumerate(sizes)]
    _check(codec, imgs, mode, s, r)


def test_mixed_layouts_in_one_call(codec):
    """Planar, 3- and 4-channel interleaved images and edge sizes in one call
    (one launch per layout class); planes are numbered image by image."""
    imgs = [(inputs.synth_image(40, 56, 1, channels=2), False),
            (np.moveaxis(inputs.synth_image(33, 70, 2, channels=3), 0, -1).copy(), True),
            (inputs.synth_image(17, 9, 3), False),
            (np.moveaxis(inputs.synth_image(64, 64, 4, channels=4), 0, -1).copy(), True),
            (np.moveaxis(inputs.synth_image(16, 24, 5, channels=3), 0, -1).copy(), True)]
    for mode, s, r in QUANTS[:4]:
        _check(codec, imgs, mode, s, r)
    _check(codec, imgs, ADCT_Q_STEP, 4, 64, with_dst=False)
    _check(codec, imgs, ADCT_Q_STEP, 4, 64, with_coef=False)


@pytest.mark.parametrize("mode,s,r", [(ADCT_Q_STEP, 4, 64), (ADCT_Q_ZONAL_ZZ, None, 6)])
def test_inverse_into_interleaved_and_edge_images(codec, mode, s, r):
    imgs = [(np.moveaxis(inputs.synth_image(45, 83, 7, channels=3), 0, -1).copy(), True),
            (np.moveaxis(inputs.synth_image(16, 16, 8, channels=4), 0, -1).copy(), True),
            (inputs.synth_image(21, 35, 9, channels=2), False),
            (np.moveaxis(inputs.synth_image(75, 93, 10, channels=3), 0, -1).copy(), True),  # split
            (inputs.synth_image(100, 61, 11, channels=1), False)]  # split
    coefs = _check(codec, imgs, mode, s, r, with_dst=False)
    q = _quant(mode, s, r)
    outs = []
    for (x, inter) in imgs:
        d, b = _pitched(np.zeros_like(x), inter)
        b.fill_(GUARD)
        outs.append((d, b))
    codec.inverse([Image(None, d, c, inter) for (d, _), c, (_, inter) in zip(outs, coefs, imgs)], q)
    torch.cuda.synchronize()
    for (x, inter), (d, b) in zip(imgs, outs):
        for k, plane in enumerate(_planes(x, inter)):
            _, rec = _ref(np.ascontiguousarray(plane), mode, s, r)
            out = d[:, :, k] if inter else d[k]
            assert np.array_equal(out.cpu().numpy(), rec)


def test_forward_and_quantise_of_interleaved(codec):
    x = np.moveaxis(inputs.synth_image(30, 50, 12, channels=3), 0, -1).copy()
    src, _ = _pitched(x, True)
    coef = _coef(3, 30, 50, ADCT_Q_STEP, 64)
    codec.forward([Image(src, None, coef, True)])
    torch.cuda.synchronize()
    for k in range(3):
        plane = np.ascontiguousarray(x[:, :, k])
        Z = oracle.forward(np.pad(plane, ((0, 2), (0, 6)), mode="edge"))
        assert np.array_equal(coef[k].cpu().numpy().astype(np.int64), Z)
    q = _quant(ADCT_Q_STEP, 4, 64)
    codec.quantise([Image(None, None, coef, True)], q)  # coefficients only: the pixel layout does not matter
    torch.cuda.synchronize()
    for k in range(3):
        qref, _ = _ref(np.ascontiguousarray(x[:, :, k]), ADCT_Q_STEP, 4, 64)
        assert np.array_equal(coef[k].cpu().numpy().astype(np.int64), qref)


def test_graph_and_noalloc_with_layouts(codec):
    q = _quant(ADCT_Q_STEP, 4, 64)
    imgs = [(np.moveaxis(inputs.synth_image(19, 37, 21, channels=3), 0, -1).copy(), True),
            (np.moveaxis(inputs.synth_image(48, 40, 22, channels=3), 0, -1).copy(), True)]
    refs = [[_ref(np.ascontiguousarray(p), ADCT_Q_STEP, 4, 64) for p in _planes(x, True)] for x, _ in imgs]
    for _ in range(2):  # capture, then replay
        ims = []
        for x, inter in imgs:
            src, _ = _pitched(x, inter)
            dst, _ = _pitched(np.zeros_like(x), inter)
            ims.append(Image(src, dst, _coef(3, x.shape[0], x.shape[1], ADCT_Q_STEP, 64), inter))
        codec.roundtrip_graph(ims, q)
        torch.cuda.synchronize()
        for im, ref in zip(ims, refs):
            for k, (qref, rec) in enumerate(ref):
                assert np.array_equal(im.coef[k].cpu().numpy().astype(np.int64), qref)
                assert np.array_equal(im.dst[:, :, k].cpu().numpy(), rec)
    lib = _native.load()
    sh = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    ims = []
    for x, inter in imgs:
        src, _ = _pitched(x, inter)
        dst, _ = _pitched(np.zeros_like(x), inter)
        ims.append(Image(src, dst, _coef(3, x.shape[0], x.shape[1], ADCT_Q_STEP, 64), inter))
    assert lib.adct_roundtrip_noalloc(image_array(ims), len(ims), ctypes.byref(q), sh) == _native.ADCT_OK
    torch.cuda.synchronize()
    for im, ref in zip(ims, refs):
        for k, (qref, rec) in enumerate(ref):
            assert np.array_equal(im.dst[:, :, k].cpu().numpy(), rec)
    # layout classes mixed in one allocation-free call: one launch each
    x = inputs.synth_image(21, 19, 1)[0]
    p, _ = _pitched(x[None], False)
    pd, _ = _pitched(np.zeros_like(x)[None], False)
    pc = _coef(1, 21, 19, ADCT_Q_STEP, 64)
    y = inputs.synth_image(16, 16, 2)[0]
    a = torch.from_numpy(y).to(DEV)
    ad, ac = torch.empty_like(a), _coef(1, 16, 16, ADCT_Q_STEP, 64)
    mixed = image_array([ims[0], Image(p, pd, pc), Image(a, ad, ac)])
    assert lib.adct_roundtrip_noalloc(mixed, 3, ctypes.byref(q), sh) == _native.ADCT_OK
    torch.cuda.synchronize()
    for out, c, plane in ((pd[0], pc[0], x), (ad, ac[0], y)):
        qref, rec = _ref(plane, ADCT_Q_STEP, 4, 64)
        assert np.array_equal(out.cpu().numpy(), rec)
        assert np.array_equal(c.cpu().numpy().astype(np.int64), qref)


def test_graph_with_split_edge_images(codec):
    """Images large enough to be split (a masked interior, then their edge
    strips launched as its programmatic dependent), captured in a CUDA graph
    and replayed, planar and interleaved in one call: equal to the oracle."""
    q = _quant(ADCT_Q_STEP, 4, 64)
    imgs = [(inputs.synth_image(75, 93, 31, channels=2), False),
            (np.moveaxis(inputs.synth_image(100, 61, 32, channels=3), 0, -1).copy(), True),
            (inputs.synth_image(72, 93, 33, channels=1), False)]
    refs = [[_ref(np.ascontiguousarray(p), ADCT_Q_STEP, 4, 64) for p in _planes(x, inter)] for x, inter in imgs]
    for _ in range(3):  # capture, then replay twice
        ims = []
        for x, inter in imgs:
            src, _ = _pitched(x, inter)
            dst, _ = _pitched(np.zeros_like(x), inter)
            C = x.shape[2] if inter else x.shape[0]
            H, W = (x.shape[0], x.shape[1]) if inter else (x.shape[1], x.shape[2])
            ims.append(Image(src, dst, _coef(C, H, W, ADCT_Q_STEP, 64), inter))
        codec.roundtrip_graph(ims, q)
        torch.cuda.synchronize()
        for im, ref, (x, inter) in zip(ims, refs, imgs):
            for k, (qref, rec) in enumerate(ref):
                assert np.array_equal(im.coef[k].cpu().numpy().astype(np.int64), qref)
                out = im.dst[:, :, k] if inter else im.dst[k]
                assert np.array_equal(out.cpu().numpy(), rec)


def test_layout_errors(codec):
    q = _quant(ADCT_Q_STEP, 4, 64)
    two = torch.zeros((16, 16, 2), dtype=torch.uint8, device=DEV)
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(two, torch.zeros_like(two), None, True)], q)
    assert e.value.status == _native.ADCT_ERR_UNSUPPORTED
    odd = torch.zeros((12, 16), dtype=torch.uint8, device=DEV)[:, :12]
    with pytest.raises(AdctError) as e:
        codec.quality_dct([Image(odd)], 10)
    assert e.value.status == _native.ADCT_ERR_UNSUPPORTED
    hwc = torch.zeros((16, 16, 3), dtype=torch.uint8)
    with pytest.raises(AdctError) as e:
        codec.roundtrip_host([Image(hwc, hwc.clone(), None, True)], q)
    assert e.value.status == _native.ADCT_ERR_UNSUPPORTED
    narrow = torch.zeros((8, 20), dtype=torch.uint8, device=DEV)[:, :10]  # pitch 20: not a multiple of 8
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(narrow, None, torch.zeros((1, 1, 2, 8, 8), dtype=torch.int16, device=DEV))], q)
    assert e.value.status == _native.ADCT_ERR_ALIGN


def test_large_interleaved_edge_image_sampled(codec):
    """An interleaved 11999 x 65535 x 3 image (2.4 GB: pixel offsets past 2^31
    bytes, an edge block at the end of every block row and in the last block
    row), step s = 4, on sampled blocks of every channel: the oracle runs on
    the block alone, edge-extended like the image."""
    H, W = 11999, 65535
    pitch = (W * 3 + 7) // 8 * 8
    g = torch.Generator(device=DEV)
    g.manual_seed(1703)
    buf = torch.randint(0, 256, (H, pitch), dtype=torch.uint8, device=DEV, generator=g)
    src = buf[:, :W * 3].view(H, W, 3)
    out = torch.empty_like(buf)
    dst = out[:, :W * 3].view(H, W, 3)
    hb, wb = (H + 7) // 8, (W + 7) // 8
    coef = torch.empty((3, hb, wb, 8, 8), dtype=torch.int16, device=DEV)
    Qt = inputs.step_table(4)
    codec.roundtrip([Image(src, dst, coef, True)], make_quant(ADCT_Q_STEP, Qt))
    torch.cuda.synchronize()
    rng = np.random.default_rng(8)
    picks = [(hb - 1, wb - 1), (hb - 1, 0), (0, wb - 1), (0, 0), (hb - 2, wb - 1), (hb - 1, wb - 2)]
    picks += [(int(rng.integers(hb)), int(rng.integers(wb))) for _ in range(40)]
    for by, bx in picks:
        y0, x0 = 8 * by, 8 * bx
        vr, vc = min(8, H - y0), min(8, W - x0)
        blk = src[y0:y0 + vr, x0:x0 + vc].cpu().numpy()
        got = dst[y0:y0 + vr, x0:x0 + vc].cpu().numpy()
        cf = coef[:, by, bx].cpu().numpy().astype(np.int64)
        for c in range(3):
            padded = np.pad(blk[:, :, c], ((0, 8 - vr), (0, 8 - vc)), mode="edge")
            q_ref, rec_ref = oracle.roundtrip(padded, oracle.MODE_STEP, Qt, 64)
            assert np.array_equal(got[:, :, c], rec_ref[:vr, :vc]), (by, bx, c)
            assert np.array_equal(cf[c], q_ref[0, 0]), (by, bx, c)
    del buf, out, coef
    torch.cuda.empty_cache()


def test_full_hd_rgb_batch_sampled(codec):
    """16 interleaved 1080x1920x3 images in one launch, sampled channels
    against the oracle (the 1080-row edge is a multiple of 8; 1917 columns
    exercise the right edge on every block row)."""
    n, H, W = 16, 1080, 1917
    pitch = (W * 3 + 7) // 8 * 8
    buf = torch.empty((n, H, pitch), dtype=torch.uint8, device=DEV)
    src = buf[:, :, :W * 3].view(n, H, W, 3)
    host = [np.moveaxis(inputs.synth_image(H, W, 500 + k, channels=3), 0, -1) for k in (0, 9, 15)]
    for k in range(n):
        src[k].copy_(torch.from_numpy(np.ascontiguousarray(np.moveaxis(
            inputs.synth_image(H, W, 500 + k, channels=3), 0, -1))))
    dst = torch.empty_like(buf)[:, :, :W * 3].view(n, H, W, 3)
    coef = torch.empty((n, 3, H // 8, (W + 7) // 8, 8, 8), dtype=torch.int16, device=DEV)
    q = _quant(ADCT_Q_STEP, 4, 64)
    codec.roundtrip([Image(src[k], dst[k], coef[k], True) for k in range(n)], q)
    torch.cuda.synchronize()
    for x, k in zip(host, (0, 9, 15)):
        for c in (0, 2):
            qref, rec = _ref(np.ascontiguousarray(x[:, :, c]), ADCT_Q_STEP, 4, 64)
            assert np.array_equal(dst[k, :, :, c].cpu().numpy(), rec)
            assert np.array_equal(coef[k, c].cpu().numpy().astype(np.int64), qref)
