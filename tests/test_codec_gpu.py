"""GPU parity of the integer codec against the oracle, bit for bit.

All calls go through the C ABI (libadct.so) via the ctypes binding.  Sizes span
several warps' chunks and ragged tails; the full-size uniform batch is checked
on every image (the oracle runs in threads on the host cores) plus an any-size
property (identity round trip)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import inputs
from paper_1702_00817_gb300.codec import (ADCT_Q_NONE, ADCT_Q_STEP, ADCT_Q_STEP_ZONAL, ADCT_Q_ZONAL, AdctError,
                                          Codec, Image, make_quant)

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
MODES = {ADCT_Q_NONE: oracle.MODE_NONE, ADCT_Q_STEP: oracle.MODE_STEP, ADCT_Q_ZONAL: oracle.MODE_ZONAL,
         ADCT_Q_STEP_ZONAL: oracle.MODE_STEP_ZONAL}


@pytest.fixture(scope="module")
def codec():
    import __graft_entry__
    __graft_entry__.build()
    c = Codec(0)
    yield c
    c.close()


def _dev_img(plane: np.ndarray):
    src = torch.from_numpy(np.ascontiguousarray(plane)).to(DEV)
    return src


def _coef_like(src: torch.Tensor):
    C = 1 if src.dim() == 2 else src.shape[0]
    H, W = src.shape[-2], src.shape[-1]
    return torch.empty((C, H // 8, W // 8, 8, 8), dtype=torch.int16, device=DEV)


def _oracle_planes(img: np.ndarray):
    return [img] if img.ndim == 2 else [img[c] for c in range(img.shape[0])]


def _check_roundtrip(codec, imgs, mode, Q=None, r=64):
    """Round trip a list of numpy images ([H,W] or [C,H,W]) in one call; compare to the oracle."""
    srcs = [_dev_img(x) for x in imgs]
    dsts = [torch.full_like(s, 7) for s in srcs]
    coefs = [_coef_like(s) for s in srcs]
    q = make_quant(mode, Q, r)
    codec.roundtrip([Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)], q)
    torch.cuda.synchronize()
    for x, d, c in zip(imgs, dsts, coefs):
        rec = d.cpu().numpy()
        cf = c.cpu().numpy().astype(np.int64)
        for k, plane in enumerate(_oracle_planes(x)):
            q_ref, rec_ref = oracle.roundtrip(plane, MODES[mode], Q, r)
            assert np.array_equal(cf[k], q_ref)
            assert np.array_equal(rec if x.ndim == 2 else rec[k], rec_ref)


def test_config1_512_step4(codec):
    img = inputs.synth_image(512, 512, inputs.BASE_SEED)[0]
    _check_roundtrip(codec, [img], ADCT_Q_STEP, inputs.step_table(4))


@pytest.mark.parametrize("s", [1, 4, 16])
def test_step_tables(codec, s):
    imgs = [inputs.synth_image(136, 200, 100 + s)[0], inputs.synth_image(64, 72, 200 + s)[0]]
    _check_roundtrip(codec, imgs, ADCT_Q_STEP, inputs.step_table(s))


@pytest.mark.parametrize("r", [0, 1, 6, 10, 16, 25, 45, 64])
def test_zonal(codec, r):
    imgs = [inputs.synth_image(120, 248, 300 + r)[0]]
    _check_roundtrip(codec, imgs, ADCT_Q_ZONAL, None, r)


def test_none_and_step_zonal(codec):
    img = inputs.synth_image(96, 160, 5)[0]
    _check_roundtrip(codec, [img], ADCT_Q_NONE)
    _check_roundtrip(codec, [img], ADCT_Q_STEP_ZONAL, inputs.step_table(4), 10)


def test_random_and_extreme_q_tables(codec):
    rng = np.random.default_rng(9)
    img = inputs.synth_image(64, 128, 6)[0]
    for Q in (np.ones(64, np.uint16), np.full(64, 65535, np.uint16), np.full(64, 2, np.uint16),
              rng.integers(1, 65536, 64).astype(np.uint16), rng.integers(1, 40, 64).astype(np.uint16)):
        _check_roundtrip(codec, [img], ADCT_Q_STEP, Q)


def test_extreme_images(codec):
    yy, xx = np.mgrid[0:64, 0:64]
    imp = np.full((64, 64), 128, np.uint8)
    imp[3, 5] = 255
    imp[40, 17] = 0
    imgs = [np.zeros((64, 64), np.uint8), np.full((64, 64), 255, np.uint8),
            (((yy + xx) % 2) * 255).astype(np.uint8), (((yy // 8 + xx // 8) % 2) * 255).astype(np.uint8), imp,
            np.random.default_rng(3).integers(0, 256, (64, 64), dtype=np.uint8)]
    for mode, Q in ((ADCT_Q_STEP, inputs.step_table(1)), (ADCT_Q_NONE, None), (ADCT_Q_STEP, inputs.step_table(16))):
        _check_roundtrip(codec, imgs, mode, Q)


def test_degenerate_shapes(codec):
    imgs = [inputs.synth_image(8, 8, 1)[0], inputs.synth_image(8, 4096, 2)[0], inputs.synth_image(4096, 8, 3)[0],
            inputs.synth_image(24, 8, 4)[0]]
    _check_roundtrip(codec, imgs, ADCT_Q_STEP, inputs.step_table(4))


def test_maximum_sides_and_64bit_offsets(codec):
    """The longest sides the ABI accepts (65536) against the oracle in full,
    and a 40000 x 65536 image (2.6 GB of pixels, 5.2 GB of coefficients) whose
    byte offsets pass 2^31 on sampled blocks: every 8x8 block is independent,
    so the oracle runs on the block alone; the samples include the four
    corner blocks."""
    _check_roundtrip(codec, [inputs.synth_image(8, 65536, 5)[0], inputs.synth_image(65536, 8, 6)[0]], ADCT_Q_STEP,
                     inputs.step_table(4))
    H, W = 40000, 65536
    g = torch.Generator(device=DEV)
    g.manual_seed(1702)
    src = torch.randint(0, 256, (H, W), dtype=torch.uint8, device=DEV, generator=g)
    dst = torch.empty_like(src)
    coef = torch.empty((1, H // 8, W // 8, 8, 8), dtype=torch.int16, device=DEV)
    Qt = inputs.step_table(4)
    codec.roundtrip([Image(src, dst, coef)], make_quant(ADCT_Q_STEP, Qt))
    torch.cuda.synchronize()
    hb, wb = H // 8, W // 8
    rng = np.random.default_rng(7)
    picks = [(hb - 1, wb - 1), (hb - 1, 0), (0, wb - 1), (0, 0)]
    picks += [(int(rng.integers(hb)), int(rng.integers(wb))) for _ in range(60)]
    for by, bx in picks:
        blk = src[8 * by:8 * by + 8, 8 * bx:8 * bx + 8].cpu().numpy()
        q_ref, rec_ref = oracle.roundtrip(blk, oracle.MODE_STEP, Qt, 64)
        assert np.array_equal(dst[8 * by:8 * by + 8, 8 * bx:8 * bx + 8].cpu().numpy(), rec_ref), (by, bx)
        assert np.array_equal(coef[0, by, bx].cpu().numpy().astype(np.int64), q_ref[0, 0]), (by, bx)
    del src, dst, coef
    torch.cuda.empty_cache()


def test_ragged_multichannel_batch_one_launch(codec):
    sizes = inputs.ragged_sizes(12, seed=11, lo_log2=3.0, hi_log2=8.0)
    imgs = inputs.ragged_batch(sizes, channels=3, base_seed=50)
    _check_roundtrip(codec, imgs, ADCT_Q_STEP, inputs.step_table(4))
    _check_roundtrip(codec, imgs, ADCT_Q_ZONAL, None, 6)


def test_split_stages_equal_oracle_and_fused(codec):
    img = inputs.synth_image(200, 264, 77)[0]
    Q = inputs.step_table(4)
    src = _dev_img(img)
    coef = _coef_like(src)
    dst = torch.empty_like(src)
    codec.forward([Image(src, None, coef)])
    torch.cuda.synchronize()
    Z = coef.cpu().numpy()[0].astype(np.int64)
    assert np.array_equal(Z, oracle.forward(img))
    q = make_quant(ADCT_Q_STEP, Q)
    codec.quantise([Image(None, None, coef)], q)
    torch.cuda.synchronize()
    qv = coef.cpu().numpy()[0].astype(np.int64)
    assert np.array_equal(qv, oracle.quantise(Z, oracle.MODE_STEP, Q))
    codec.inverse([Image(None, dst, coef)], q)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), oracle.inverse(qv, oracle.MODE_STEP, Q))
    # zonal quantise and inverse split
    codec.forward([Image(src, None, coef)])
    qz = make_quant(ADCT_Q_ZONAL, None, 10)
    codec.quantise([Image(None, None, coef)], qz)
    codec.inverse([Image(None, dst, coef)], qz)
    torch.cuda.synchronize()
    q_ref, rec_ref = oracle.roundtrip(img, oracle.MODE_ZONAL, None, 10)
    assert np.array_equal(coef.cpu().numpy()[0].astype(np.int64), q_ref)
    assert np.array_equal(dst.cpu().numpy(), rec_ref)


def test_quantise_edges_on_coefficient_input(codec):
    # quantiser on coefficients given directly: |Z| up to 8192, steps around
    # the 16384 boundary (a tie at |Z| = 8192, Q = 16384 rounds away from zero)
    rng = np.random.default_rng(12)
    edges = np.array([0, 1, -1, 2, -2, 8191, -8191, 8192, -8192, 4096, -4096, 3, -3], np.int64)
    Z = rng.integers(-8192, 8193, size=(4, 8, 8, 8)).astype(np.int64)
    Z.reshape(-1)[: edges.size] = edges
    Z[0, 1, 0, :] = 8192
    Z[0, 1, 1, :] = -8192
    for Q in (np.array([1, 2, 3, 4, 16383, 16384, 16385, 65535] * 8, np.uint16),
              rng.integers(1, 65536, 64).astype(np.uint16), inputs.step_table(1)):
        for mode in (ADCT_Q_STEP, ADCT_Q_STEP_ZONAL):
            coef = torch.from_numpy(Z.astype(np.int16).reshape(1, 4, 8, 8, 8)).to(DEV)
            codec.quantise([Image(None, None, coef)], make_quant(mode, Q, 21))
            torch.cuda.synchronize()
            expect = oracle.quantise(Z, MODES[mode], Q, 21)
            assert np.array_equal(coef.cpu().numpy()[0].astype(np.int64), expect)


def test_inverse_on_random_quantised_coefficients(codec):
    # any q with |q Q| <= 16384 (the range the quantiser produces) inverts exactly
    rng = np.random.default_rng(13)
    for Q in (inputs.step_table(1), inputs.step_table(16), rng.integers(1, 300, 64).astype(np.uint16),
              np.ones(64, np.uint16)):
        lim = (16384 // Q.reshape(-1).astype(np.int64)).reshape(8, 8)
        q = rng.integers(-lim, lim + 1, size=(6, 9, 8, 8)).astype(np.int64)
        coef = torch.from_numpy(q.astype(np.int16).reshape(1, 6, 9, 8, 8)).to(DEV)
        dst = torch.empty((48, 72), dtype=torch.uint8, device=DEV)
        codec.inverse([Image(None, dst, coef)], make_quant(ADCT_Q_STEP, Q))
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), oracle.inverse(q, oracle.MODE_STEP, Q))


def test_pitched_and_aliased_images(codec):
    img = inputs.synth_image(3 * 64, 136, 8)  # [1, 192, 136]
    big = torch.zeros((3, 80, 160), dtype=torch.uint8, device=DEV)  # pitch 160, plane stride 80*160
    planes = [inputs.synth_image(64, 136, 60 + c)[0] for c in range(3)]
    for c in range(3):
        big[c, :64, :136] = torch.from_numpy(planes[c]).to(DEV)
    view = big[:, :64, :136]
    coef = torch.empty((3, 8, 17, 8, 8), dtype=torch.int16, device=DEV)
    Q = inputs.step_table(4)
    # dst aliases src: in-place reconstruction
    codec.roundtrip([Image(view, view, coef)], make_quant(ADCT_Q_STEP, Q))
    torch.cuda.synchronize()
    out = big.cpu().numpy()
    for c in range(3):
        q_ref, rec_ref = oracle.roundtrip(planes[c], oracle.MODE_STEP, Q)
        assert np.array_equal(out[c, :64, :136], rec_ref)
        assert np.array_equal(coef.cpu().numpy()[c].astype(np.int64), q_ref)
        assert not out[c, 64:, :].any() and not out[c, :, 136:].any()  # padding untouched
    del img


def test_coef_only_and_pixels_only(codec):
    img = inputs.synth_image(72, 80, 12)[0]
    Q = inputs.step_table(16)
    q_ref, rec_ref = oracle.roundtrip(img, oracle.MODE_STEP, Q)
    src = _dev_img(img)
    coef = _coef_like(src)
    codec.roundtrip([Image(src, None, coef)], make_quant(ADCT_Q_STEP, Q))
    dst = torch.empty_like(src)
    codec.roundtrip([Image(src, dst, None)], make_quant(ADCT_Q_STEP, Q))
    torch.cuda.synchronize()
    assert np.array_equal(coef.cpu().numpy()[0].astype(np.int64), q_ref)
    assert np.array_equal(dst.cpu().numpy(), rec_ref)


def test_guard_bands_untouched(codec):
    img = inputs.synth_image(64, 64, 13)[0]
    n = 64 * 64
    band = 4096
    pix = torch.full((2 * band + n,), 0xA5, dtype=torch.uint8, device=DEV)
    out = torch.full((2 * band + n,), 0x5A, dtype=torch.uint8, device=DEV)
    cf = torch.full((2 * band + n,), 0x1234, dtype=torch.int16, device=DEV)
    pix[band:band + n] = torch.from_numpy(img.reshape(-1)).to(DEV)
    codec.roundtrip([Image(pix[band:band + n].view(64, 64), out[band:band + n].view(64, 64),
                           cf[band:band + n].view(1, 8, 8, 8, 8))], make_quant(ADCT_Q_STEP, inputs.step_table(4)))
    torch.cuda.synchronize()
    o, c = out.cpu().numpy(), cf.cpu().numpy()
    assert (o[:band] == 0x5A).all() and (o[band + n:] == 0x5A).all()
    assert (c[:band] == 0x1234).all() and (c[band + n:] == 0x1234).all()


def test_empty_batch_is_a_no_op(codec):
    codec.roundtrip([], make_quant(ADCT_Q_STEP, inputs.step_table(4)))
    codec.forward([])


def test_argument_errors(codec):
    src = torch.zeros((16, 65544), dtype=torch.uint8, device=DEV)  # wider than 65536
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(src, src.clone(), None)], make_quant(ADCT_Q_NONE))
    assert e.value.status == 2
    src = torch.zeros((16, 20), dtype=torch.uint8, device=DEV)  # rows 20 bytes apart: not 8-byte aligned
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(src, src.clone(), None)], make_quant(ADCT_Q_NONE))
    assert e.value.status == 3
    src = torch.zeros((16, 16), dtype=torch.uint8, device=DEV)
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(src, src.clone(), None)], make_quant(ADCT_Q_STEP, np.zeros(64)))
    assert e.value.status == 1
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(src, src.clone(), None)], make_quant(ADCT_Q_ZONAL, None, 65))
    assert e.value.status == 1
    raw = torch.zeros(16 * 16 + 1, dtype=torch.uint8, device=DEV)
    with pytest.raises(AdctError) as e:
        codec.roundtrip([Image(raw[1:].view(16, 16), src, None)], make_quant(ADCT_Q_NONE))
    assert e.value.status == 3
    with pytest.raises(AdctError) as e:
        codec.forward([Image(src, None, None)])
    assert e.value.status == 1


def test_graph_replay_equals_eager(codec):
    sizes = inputs.ragged_sizes(6, seed=21, lo_log2=4.0, hi_log2=8.0)
    Q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    for rep in range(3):
        imgs = inputs.ragged_batch(sizes, channels=3, base_seed=1000 * rep)
        srcs = [_dev_img(x) for x in imgs]
        dsts = [torch.empty_like(s) for s in srcs]
        coefs = [_coef_like(s) for s in srcs]
        replayed = codec.roundtrip_graph([Image(s, d, c) for s, d, c in zip(srcs, dsts, coefs)], Q)
        assert replayed == (rep > 0)
        dsts2 = [torch.empty_like(s) for s in srcs]
        coefs2 = [_coef_like(s) for s in srcs]
        codec.roundtrip([Image(s, d, c) for s, d, c in zip(srcs, dsts2, coefs2)], Q)
        torch.cuda.synchronize()
        for a, b in zip(dsts, dsts2):
            assert torch.equal(a, b)
        for a, b in zip(coefs, coefs2):
            assert torch.equal(a, b)
    # one image checked against the oracle
    q_ref, rec_ref = oracle.roundtrip(imgs[0][1], oracle.MODE_STEP, inputs.step_table(4))
    assert np.array_equal(dsts[0].cpu().numpy()[1], rec_ref)


def test_autotune_keeps_results(codec):
    imgs = [inputs.synth_image(256, 256, 30 + k)[0] for k in range(4)]
    srcs = [_dev_img(x) for x in imgs]
    dsts = [torch.empty_like(s) for s in srcs]
    Q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    before = codec.get_launch()
    best, us = codec.autotune([Image(s, d, None) for s, d in zip(srcs, dsts)], Q, reps=2)
    assert us > 0 and best["threads_per_cta"] in (32, 64, 96, 128)
    codec.roundtrip([Image(s, d, None) for s, d in zip(srcs, dsts)], Q)
    torch.cuda.synchronize()
    for x, d in zip(imgs, dsts):
        assert np.array_equal(d.cpu().numpy(), oracle.roundtrip(x, oracle.MODE_STEP, inputs.step_table(4))[1])
    codec.set_launch(before["threads_per_cta"], before["ctas_per_sm"] or -1, before["stage_coef"])


def test_launch_shape_automatic_default():
    c = Codec(0)
    assert c.get_launch()["ctas_per_sm"] == 0  # chosen per kernel by the library
    assert c.get_launch()["stage_coef"] == -1  # staging chosen per call by the library
    c.set_launch(64, 5, 0)
    assert c.get_launch() == {"threads_per_cta": 64, "ctas_per_sm": 5, "stage_coef": 0, "reserved": 0}
    c.set_launch(128, -1, 1)
    assert c.get_launch()["ctas_per_sm"] == 0 and c.get_launch()["stage_coef"] == 1
    c.set_launch(0, 0, -1)
    assert c.get_launch()["stage_coef"] == -1
    c.close()


def test_host_pipeline_equals_device_path(codec):
    sizes = inputs.ragged_sizes(9, seed=5, lo_log2=5.0, hi_log2=9.0)
    imgs = inputs.ragged_batch(sizes, channels=2, base_seed=7)
    Q = inputs.step_table(4)
    hs = [torch.from_numpy(x).pin_memory() for x in imgs]
    hd = [torch.empty_like(h).pin_memory() for h in hs]
    hc = [torch.empty((x.shape[0], x.shape[1] // 8, x.shape[2] // 8, 8, 8), dtype=torch.int16).pin_memory()
          for x in imgs]
    codec.roundtrip_host([Image(s, d, c) for s, d, c in zip(hs, hd, hc)], make_quant(ADCT_Q_STEP, Q),
                         chunk_bytes=200_000)
    for x, d, c in zip(imgs, hd, hc):
        for k in range(x.shape[0]):
            q_ref, rec_ref = oracle.roundtrip(x[k], oracle.MODE_STEP, Q)
            assert np.array_equal(d.numpy()[k], rec_ref)
            assert np.array_equal(c.numpy()[k].astype(np.int64), q_ref)


def test_repeated_batch_reuses_its_table_and_sees_new_pixels(codec):
    # the same tensors called again (identical descriptor table, reused without an
    # upload) must see the new pixel values; a second stream gets its own table
    Q = inputs.step_table(4)
    q = make_quant(ADCT_Q_STEP, Q)
    a = inputs.synth_image(64, 96, 500)[0]
    b = inputs.synth_image(64, 96, 501)[0]
    src = _dev_img(a)
    dst = torch.empty_like(src)
    coef = _coef_like(src)
    s2 = torch.cuda.Stream()
    for k, img in enumerate((a, b, a, b)):
        src.copy_(torch.from_numpy(img))
        stream = s2 if k == 3 else torch.cuda.current_stream()
        stream.wait_stream(torch.cuda.current_stream())
        codec.roundtrip([Image(src, dst, coef)], q, stream=stream)
        torch.cuda.current_stream().wait_stream(stream)
        torch.cuda.synchronize()
        q_ref, rec_ref = oracle.roundtrip(img, oracle.MODE_STEP, Q)
        assert np.array_equal(dst.cpu().numpy(), rec_ref)
        assert np.array_equal(coef.cpu().numpy()[0].astype(np.int64), q_ref)


def test_host_pipeline_merges_contiguous_copies(codec):
    # a contiguous host batch: consecutive images' copies are merged into few large copies
    n, H, W = 12, 72, 136
    host = np.ascontiguousarray(inputs.synth_batch(n, H, W, base_seed=300)[:, 0])
    hs = torch.from_numpy(host).pin_memory()
    hd = torch.empty_like(hs).pin_memory()
    hc = torch.empty((n, H // 8, W // 8, 8, 8), dtype=torch.int16).pin_memory()
    Q = inputs.step_table(16)
    codec.roundtrip_host([Image(hs[k], hd[k], hc[k:k + 1]) for k in range(n)], make_quant(ADCT_Q_STEP, Q),
                         chunk_bytes=5 * H * W)
    for k in (0, 4, 5, 11):
        q_ref, rec_ref = oracle.roundtrip(host[k], oracle.MODE_STEP, Q)
        assert np.array_equal(hd[k].numpy(), rec_ref)
        assert np.array_equal(hc[k].numpy().astype(np.int64), q_ref)


@pytest.mark.parametrize("mode,Q,r", [(ADCT_Q_STEP, 4, 64), (ADCT_Q_ZONAL, None, 64), (ADCT_Q_STEP, 1, 64),
                                      (ADCT_Q_ZONAL, None, 10)])
def test_full_size_uniform_batch(codec, mode, Q, r):
    """256 x 1080x1920 in the launch configuration the benchmark times: every
    image against the oracle (run in threads on the host cores), plus the
    identity property for ZONAL r = 64."""
    n, H, W = 256, 1080, 1920
    host = inputs.synth_batch(n, H, W)[:, 0]
    src = torch.from_numpy(host).to(DEV)
    dst = torch.empty_like(src)
    coef = torch.empty((n, H // 8, W // 8, 8, 8), dtype=torch.int16, device=DEV)
    Qt = inputs.step_table(Q) if Q else None
    codec.roundtrip([Image(src[k], dst[k], coef[k:k + 1]) for k in range(n)], make_quant(mode, Qt, r))
    torch.cuda.synchronize()
    if mode == ADCT_Q_ZONAL and r == 64:
        assert torch.equal(dst, src)  # nothing discarded: exact for every image
    dh, ch = dst.cpu().numpy(), coef.cpu().numpy()

    def same(k):
        q_ref, rec_ref = oracle.roundtrip(host[k], MODES[mode], Qt, r)
        return np.array_equal(dh[k], rec_ref) and np.array_equal(ch[k].astype(np.int64), q_ref)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        ok = list(ex.map(same, range(n)))
    assert all(ok), [k for k, o in enumerate(ok) if not o][:10]


def test_autotune_cache_file(codec, tmp_path):
    imgs = [inputs.synth_image(128, 192, 40 + k)[0] for k in range(3)]
    srcs = [_dev_img(x) for x in imgs]
    ims = [Image(s, torch.empty_like(s), None) for s in srcs]
    Q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    path = str(tmp_path / "tune.json")
    before = codec.get_launch()
    shape, us = codec.autotune(ims, Q, reps=1, cache=path)
    assert us is not None and us > 0 and os.path.exists(path)
    codec.set_launch(32, 2, 0)  # something else
    shape2, us2 = codec.autotune(ims, Q, reps=1, cache=path)  # a hit: nothing measured
    assert us2 is None and shape2 == shape
    got = codec.get_launch()
    assert got["threads_per_cta"] == shape["threads_per_cta"] and got["stage_coef"] == shape["stage_coef"]
    codec.roundtrip(ims, Q)
    torch.cuda.synchronize()
    for x, im in zip(imgs, ims):
        assert np.array_equal(im.dst.cpu().numpy(), oracle.roundtrip(x, oracle.MODE_STEP, inputs.step_table(4))[1])
    codec.set_launch(before["threads_per_cta"], before["ctas_per_sm"] or -1, before["stage_coef"])


def test_binding_refuses_host_tensors_for_device_calls(codec):
    src = torch.zeros((16, 16), dtype=torch.uint8)
    with pytest.raises(ValueError):
        codec.roundtrip([Image(src, torch.zeros_like(src), None)], make_quant(ADCT_Q_STEP, inputs.step_table(4)))
    dev_src = src.to(DEV)
    with pytest.raises(ValueError):
        codec.roundtrip_host([Image(dev_src, torch.zeros_like(dev_src), None)],
                             make_quant(ADCT_Q_STEP, inputs.step_table(4)))
