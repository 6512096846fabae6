"""Packed zonal coefficients (ADCT_Q_ZONAL_ZZ) against the oracle, bit for bit.

The packed layout stores, per 8x8 block, only the r coefficients the zonal
quantiser keeps (Sec. 3: the first r in zig-zag order), in that order.  The
expected values are the oracle's dense zonal q read out in the oracle's own
zig-zag order; the reconstructions are the oracle's zonal round trip."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import _native, inputs
from paper_1702_00817_gb300.codec import (ADCT_Q_ZONAL, ADCT_Q_ZONAL_ZZ, AdctError, Codec, Image, image_array,
                                          make_quant)
from paper_1702_00817_gb300.serve import NativeServer, Server

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ORDER = np.argsort(oracle.zigzag_rank().reshape(64))  # ORDER[t] = 8 i + j of zig-zag position t


@pytest.fixture(scope="module")
def codec():
    import __graft_entry__
    __graft_entry__.build()
    c = Codec(0)
    yield c
    c.close()


def _planes(img):
    return [img] if img.ndim == 2 else [img[c] for c in range(img.shape[0])]


def _packed_ref(plane, r):
    """(packed q [H/8, W/8, r] int64, reconstruction) from the oracle's zonal round trip."""
    q, rec = oracle.roundtrip(plane, oracle.MODE_ZONAL, None, r)
    hb, wb = q.shape[:2]
    return q.reshape(hb, wb, 64)[:, :, ORDER[:r]], rec


def _packed_like(img, r, fill=123):
    C = 1 if img.ndim == 2 else img.shape[0]
    return torch.full((C, img.shape[-2] // 8, img.shape[-1] // 8, r), fill, dtype=torch.int16, device=DEV)


def _check(codec, imgs, r, with_dst=True, stage_coef=1):
    srcs = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in imgs]
    dsts = [torch.full_like(s, 7) if with_dst else None for s in srcs]
    coefs = [_packed_like(x, r) for x in imgs]
    q = make_quant(ADCT_Q_ZONAL_ZZ, None, r)
    old = codec.get_launch()
    codec.set_launch(0, 0, stage_coef)
    try:
        codec.roundtrip([Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)], q)
        torch.cuda.synchronize()
    finally:
        codec.set_launch(old["threads_per_cta"], old["ctas_per_sm"] or -1, old["stage_coef"])
    for x, d, c in zip(imgs, dsts, coefs):
        cf = c.cpu().numpy().astype(np.int64)
        for k, plane in enumerate(_planes(x)):
            pref, rec_ref = _packed_ref(plane, r)
            assert np.array_equal(cf[k], pref), (r, k)
            if with_dst:
                rec = d.cpu().numpy()
                assert np.array_equal(rec if x.ndim == 2 else rec[k], rec_ref), (r, k)
    return coefs


@pytest.mark.parametrize("r", [0, 1, 3, 6, 10, 15, 25, 45, 63, 64])
def test_packed_roundtrip_ragged_multichannel(codec, r):
    """Odd r makes every other tile start on a 2-byte boundary; ragged
    multi-channel planes make tiles that span planes."""
    sizes = inputs.ragged_sizes(9, seed=30 + r, lo_log2=3.0, hi_log2=8.0)
    imgs = inputs.ragged_batch(sizes, channels=3, base_seed=60 + r)
    _check(codec, imgs, r)


@pytest.mark.parametrize("r", [1, 10, 37])
def test_packed_coefficients_only_and_direct_stores(codec, r):
    imgs = [inputs.synth_image(136, 264, 5 + r)[0], inputs.synth_image(8, 8, 6)[0], inputs.synth_image(72, 40, 7)]
    _check(codec, imgs, r, with_dst=False)
    _check(codec, imgs, r, with_dst=True, stage_coef=0)


@pytest.mark.parametrize("r", [1, 2, 10, 21, 64])
def test_packed_inverse_equals_oracle(codec, r):
    imgs = [inputs.synth_image(200, 136, 90 + r)[0], inputs.synth_image(64, 64, 91), inputs.synth_image(8, 16, 92)[0]]
    coefs = _check(codec, imgs, r, with_dst=False)
    q = make_quant(ADCT_Q_ZONAL_ZZ, None, r)
    outs = [torch.zeros(x.shape, dtype=torch.uint8, device=DEV) for x in imgs]
    codec.inverse([Image(None, o, c) for o, c in zip(outs, coefs)], q)
    torch.cuda.synchronize()
    for x, o in zip(imgs, outs):
        rec = o.cpu().numpy()
        for k, plane in enumerate(_planes(x)):
            _, rec_ref = _packed_ref(plane, r)
            assert np.array_equal(rec if x.ndim == 2 else rec[k], rec_ref)


def test_packed_inverse_of_random_coefficients(codec):
    """Any packed values in the forward range (|Z| <= 8192) decode like the
    oracle's inverse of the same values placed at their zig-zag positions."""
    rng = np.random.default_rng(4)
    r, hb, wb = 13, 17, 9
    packed = rng.integers(-8192, 8193, (1, hb, wb, r)).astype(np.int16)
    dense = np.zeros((hb, wb, 64), np.int64)
    dense[:, :, ORDER[:r]] = packed[0]
    ref = oracle.inverse(dense.reshape(hb, wb, 8, 8), oracle.MODE_ZONAL)
    out = torch.zeros((hb * 8, wb * 8), dtype=torch.uint8, device=DEV)
    codec.inverse([Image(None, out, torch.from_numpy(packed).to(DEV))], make_quant(ADCT_Q_ZONAL_ZZ, None, r))
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_packed_pixels_equal_dense_zonal(codec):
    """The layout changes the bytes stored, never the reconstruction."""
    imgs = inputs.ragged_batch(inputs.ragged_sizes(6, seed=8, lo_log2=4.0, hi_log2=9.0), channels=2, base_seed=8)
    srcs = [torch.from_numpy(x).to(DEV) for x in imgs]
    a = [torch.empty_like(s) for s in srcs]
    b = [torch.empty_like(s) for s in srcs]
    dense = [torch.empty((x.shape[0], x.shape[1] // 8, x.shape[2] // 8, 8, 8), dtype=torch.int16, device=DEV)
             for x in imgs]
    codec.roundtrip([Image(s, d, c) for s, d, c in zip(srcs, a, dense)], make_quant(ADCT_Q_ZONAL, None, 10))
    codec.roundtrip([Image(s, d, _packed_like(x, 10)) for s, d, x in zip(srcs, b, imgs)],
                    make_quant(ADCT_Q_ZONAL_ZZ, None, 10))
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_packed_graph_host_and_noalloc_paths(codec):
    r = 10
    imgs = [inputs.synth_image(120, 248, 11)[0], inputs.synth_image(64, 88, 12)[0], inputs.synth_image(256, 8, 13)[0]]
    refs = [_packed_ref(x, r) for x in imgs]
    q = make_quant(ADCT_Q_ZONAL_ZZ, None, r)
    # CUDA graph replay
    for _ in range(2):
        srcs = [torch.from_numpy(x).to(DEV) for x in imgs]
        dsts = [torch.empty_like(s) for s in srcs]
        coefs = [_packed_like(x, r) for x in imgs]
        codec.roundtrip_graph([Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)], q)
        torch.cuda.synchronize()
        for (pref, rec_ref), d, c in zip(refs, dsts, coefs):
            assert np.array_equal(c[0].cpu().numpy().astype(np.int64), pref)
            assert np.array_equal(d.cpu().numpy(), rec_ref)
    # host buffers: one chunk per image, then all images in one chunk (the
    # packed images are not multiples of 16 bytes, so the staging pads them)
    for chunk in (1, 64 << 20):
        hs = [torch.from_numpy(x).pin_memory() for x in imgs]
        hd = [torch.empty_like(h).pin_memory() for h in hs]
        hc = [torch.full((1, x.shape[0] // 8, x.shape[1] // 8, r), 5, dtype=torch.int16).pin_memory() for x in imgs]
        codec.roundtrip_host([Image(s, d, c) for s, d, c in zip(hs, hd, hc)], q, chunk_bytes=chunk)
        for (pref, rec_ref), d, c in zip(refs, hd, hc):
            assert np.array_equal(c[0].numpy().astype(np.int64), pref)
            assert np.array_equal(d.numpy(), rec_ref)
    # the allocation-free entry point
    lib = _native.load()
    srcs = [torch.from_numpy(x).to(DEV) for x in imgs]
    dsts = [torch.empty_like(s) for s in srcs]
    coefs = [_packed_like(x, r) for x in imgs]
    arr = image_array([Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)], q)
    sh = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    assert lib.adct_roundtrip_noalloc(arr, len(imgs), ctypes.byref(q), sh) == _native.ADCT_OK
    torch.cuda.synchronize()
    for (pref, rec_ref), d, c in zip(refs, dsts, coefs):
        assert np.array_equal(c[0].cpu().numpy().astype(np.int64), pref)
        assert np.array_equal(d.cpu().numpy(), rec_ref)


def test_packed_quantise_is_unsupported(codec):
    packed = torch.zeros((1, 2, 2, 2), dtype=torch.int16, device=DEV)
    with pytest.raises(AdctError) as e:
        codec.quantise([Image(None, None, packed)], make_quant(ADCT_Q_ZONAL_ZZ, None, 2))
    assert e.value.status == _native.ADCT_ERR_UNSUPPORTED


@pytest.mark.parametrize("server_cls", [Server, NativeServer])
def test_servers_store_packed_coefficients(server_cls):
    r = 6
    q = make_quant(ADCT_Q_ZONAL_ZZ, None, r)
    imgs = [torch.from_numpy(inputs.synth_image(h, w, 70 + h)[0]).pin_memory() for h, w in ((256, 256), (64, 520))]
    srv = server_cls(0, budget_bytes=64 << 20, streams=2, quant=q)
    try:
        enc = [srv.encode(px) for px in imgs]
        for e in enc:
            assert e.done.wait(30) and e.error is None
        dec = [srv.decode(e.result) for e in enc]
        for d in dec:
            assert d.done.wait(30) and d.error is None
        for px, e, d in zip(imgs, enc, dec):
            pref, rec_ref = _packed_ref(px.numpy(), r)
            assert np.array_equal(d.result.numpy(), rec_ref)
            if server_cls is Server:
                stored = srv.store.get(e.result)["coef"]
                assert stored.numel() == pref.size
                assert np.array_equal(stored[0].cpu().numpy().astype(np.int64), pref)
    finally:
        srv.close()


def test_full_size_packed_sampled(codec):
    """256 x 1080x1920 with r = 10 in the benchmark's launch configuration:
    sampled images against the oracle."""
    n, H, W, r = 256, 1080, 1920, 10
    host = inputs.synth_batch(n, H, W)[:, 0]
    src = torch.from_numpy(host).to(DEV)
    dst = torch.empty_like(src)
    coef = torch.empty((n, H // 8, W // 8, r), dtype=torch.int16, device=DEV)
    codec.roundtrip([Image(src[k], dst[k], coef[k:k + 1]) for k in range(n)], make_quant(ADCT_Q_ZONAL_ZZ, None, r))
    torch.cuda.synchronize()
    for k in (0, 1, 128, 255):
        pref, rec_ref = _packed_ref(host[k], r)
        assert np.array_equal(dst[k].cpu().numpy(), rec_ref)
        assert np.array_equal(coef[k].cpu().numpy().astype(np.int64), pref)


def test_every_r_every_zonal_kind(codec):
    """r = 0..64 covers every zone the kernels are specialised on and both
    sides of each zone boundary: dense and packed round trips, pixels only,
    packed coefficients only, the packed inverse and the squared error."""
    imgs = [inputs.synth_image(40, 264, 3)[0], inputs.synth_image(24, 16, 4, channels=3)]
    srcs = [torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in imgs]
    for r in range(65):
        refs = [[_packed_ref(p, r) for p in _planes(x)] for x in imgs]
        dense_ref = [[oracle.roundtrip(p, oracle.MODE_ZONAL, None, r)[0] for p in _planes(x)] for x in imgs]
        dz, pz = make_quant(ADCT_Q_ZONAL, None, r), make_quant(ADCT_Q_ZONAL_ZZ, None, r)
        dense = [torch.empty((1 if x.ndim == 2 else x.shape[0], x.shape[-2] // 8, x.shape[-1] // 8, 8, 8),
                             dtype=torch.int16, device=DEV) for x in imgs]
        d1 = [torch.empty_like(s) for s in srcs]
        codec.roundtrip([Image(s, d, c) for s, d, c in zip(srcs, d1, dense)], dz)
        d2 = [torch.empty_like(s) for s in srcs]
        codec.roundtrip([Image(s, d) for s, d in zip(srcs, d2)], pz)
        d3 = [torch.empty_like(s) for s in srcs]
        codec.roundtrip([Image(s, d) for s, d in zip(srcs, d3)], dz)
        sse = codec.quality([Image(s) for s in srcs], dz).cpu().numpy()
        if r > 0:
            packed = [_packed_like(x, r) for x in imgs]
            codec.roundtrip([Image(s, None, c) for s, c in zip(srcs, packed)], pz)
            d4 = [torch.empty_like(s) for s in srcs]
            codec.inverse([Image(None, d, c) for d, c in zip(d4, packed)], pz)
        torch.cuda.synchronize()
        plane = 0
        for m, x in enumerate(imgs):
            for k, p in enumerate(_planes(x)):
                pref, rec_ref = refs[m][k]
                pick = (lambda t: t.cpu().numpy()) if x.ndim == 2 else (lambda t, k=k: t[k].cpu().numpy())
                assert np.array_equal(dense[m][k].cpu().numpy().astype(np.int64), dense_ref[m][k]), r
                for out in (d1, d2, d3):
                    assert np.array_equal(pick(out[m]), rec_ref), r
                assert int(sse[plane]) == oracle.sse(rec_ref, p), r
                if r > 0:
                    assert np.array_equal(packed[m][k].cpu().numpy().astype(np.int64), pref), r
                    assert np.array_equal(pick(d4[m]), rec_ref), r
                plane += 1
