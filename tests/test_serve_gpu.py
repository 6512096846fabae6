"""Continuous-batching server: results in the mix equal results alone, requests
overlap on the device, admission respects the device-memory budget."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1702_00817_gb300 import inputs
from paper_1702_00817_gb300.codec import ADCT_Q_STEP, Codec, Image, make_quant
from paper_1702_00817_gb300.serve import NativeServer, Request, Server, poisson_run

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
SIZES = [(256, 256), (512, 512), (1080, 1920), (256, 512)]


@pytest.fixture(scope="module")
def images():
    import __graft_entry__
    __graft_entry__.build()
    return {hw: [torch.from_numpy(inputs.synth_image(hw[0], hw[1], 40 + k)[0]).pin_memory() for k in range(2)]
            for hw in SIZES}


def _alone(codec, px, q):
    """Encode then decode one image on its own (synchronously)."""
    src = px.to(DEV)
    coef = torch.empty((1, src.shape[0] // 8, src.shape[1] // 8, 8, 8), dtype=torch.int16, device=DEV)
    dst = torch.empty_like(src)
    codec.roundtrip([Image(src, None, coef)], q)
    codec.inverse([Image(None, dst, coef)], q)
    torch.cuda.synchronize()
    return coef.cpu(), dst.cpu()


@pytest.mark.parametrize("server_cls", [Server, NativeServer])
def test_results_in_the_mix_equal_results_alone(images, server_cls):
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    srv = server_cls(0, budget_bytes=1 << 30, streams=3, quant=q)
    try:
        enc = [srv.encode(images[hw][k]) for hw in SIZES for k in range(2)]
        for r in enc:
            assert r.done.wait(30) and r.error is None
        dec = [srv.decode(r.result) for r in enc] + [srv.encode(images[SIZES[0]][0])]
        for r in dec:
            assert r.done.wait(30) and r.error is None
        codec = Codec(0)
        for e, d in zip(enc, dec):
            coef_ref, px_ref = _alone(codec, e.pixels, q)
            if server_cls is Server:
                assert torch.equal(srv.store.get(e.result)["coef"].cpu(), coef_ref)
            assert torch.equal(d.result, px_ref)
        # and against the oracle for one image
        q_ref, rec_ref = oracle.roundtrip(images[SIZES[1]][0].numpy(), oracle.MODE_STEP, inputs.step_table(4))
        assert np.array_equal(dec[2].result.numpy(), rec_ref)
        codec.close()
    finally:
        srv.close()


@pytest.mark.parametrize("server_cls", [Server, NativeServer])
def test_requests_overlap_and_stream_admits_mid_flight(images, server_cls):
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    srv = server_cls(0, budget_bytes=2 << 30, streams=4, quant=q)
    try:
        by_size = {hw: images[hw] for hw in SIZES}
        reqs = poisson_run(srv, rate=3000.0, n_requests=300, sizes=SIZES, images_by_size=by_size, seed=3,
                           warm_handles=8)
        assert all(r.done.is_set() and r.error is None for r in reqs)
        stats = srv.stats
        assert stats["max_overlap"] >= 2          # batches were in flight together
        assert stats["launches"] < len(reqs) + 8   # requests were batched
        # some request was admitted before an earlier one completed
        reqs.sort(key=lambda r: r.t_arrival)
        assert any(b.t_admit < a.t_done for a, b in zip(reqs, reqs[1:]))
        lat = np.array([r.latency for r in reqs])
        assert np.all(lat > 0)
    finally:
        srv.close()


def test_budget_rejects_oversized_and_evicts_old_entries(images):
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    small = 3 * 512 * 512 + 10
    srv = Server(0, budget_bytes=small, streams=2, quant=q)
    try:
        big = srv.encode(images[(1080, 1920)][0])
        assert big.done.wait(30) and big.error is not None and "budget" in big.error
        a = srv.encode(images[(256, 256)][0])
        assert a.done.wait(30) and a.error is None
        b = srv.encode(images[(512, 512)][0])  # needs more than is left: evicts a
        assert b.done.wait(30) and b.error is None
        assert srv.store.get(a.result) is None and srv.stats["evicted"] >= 1
        lost = srv.decode(a.result)
        assert lost.done.wait(30) and lost.error == "unknown handle"
        ok = srv.decode(b.result)
        assert ok.done.wait(30) and ok.error is None
        assert srv.in_flight_bytes == 0 and srv.store.bytes <= small
    finally:
        srv.close()


def test_native_budget_rejects_oversized_and_evicts_old_entries(images):
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    small = 3 * 512 * 512 + 4096
    srv = NativeServer(0, budget_bytes=small, streams=2, quant=q)
    try:
        big = srv.encode(images[(1080, 1920)][0])
        assert big.done.wait(30) and big.error == "ADCT_ERR_OOM"
        a = srv.encode(images[(256, 256)][0])
        assert a.done.wait(30) and a.error is None
        b = srv.encode(images[(512, 512)][0])  # needs the space a holds: a is evicted
        assert b.done.wait(30) and b.error is None
        assert srv.stats["evicted"] >= 1 and srv.stats["oversized"] == 1
        lost = srv.decode(a.result)
        assert lost.done.wait(30) and lost.error == "unknown handle"
        ok = srv.decode(b.result)
        assert ok.done.wait(30) and ok.error is None
        codec = Codec(0)
        assert torch.equal(ok.result, _alone(codec, images[(512, 512)][0], q)[1])
        codec.close()
    finally:
        srv.close()


def test_native_clock_is_the_perf_counter_clock():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1702_00817_gb300 import _native
    lib = _native.load()
    t0 = time.perf_counter()
    tn = lib.adct_server_clock()
    t1 = time.perf_counter()
    assert t0 - 1e-3 <= tn <= t1 + 1e-3


@pytest.mark.parametrize("server_cls", [Server, NativeServer])
def test_cancel_withdraws_queued_requests(images, server_cls):
    """Requests queued behind a memory-bound backlog can be withdrawn: they
    complete as cancelled and never run; the others complete normally, every
    request exactly once, and nothing stays pinned or allocated."""
    q = make_quant(ADCT_Q_STEP, inputs.step_table(4))
    big = images[(1080, 1920)][0]
    srv = server_cls(0, budget_bytes=16 << 20, streams=2, quant=q)  # room for two encodes at a time
    try:
        reqs = [srv.encode(big) for _ in range(24)]
        flags = [srv.cancel(r) for r in reqs[8:]]
        for r in reqs:
            assert r.done.wait(60)
        cancelled = [r for r in reqs if r.error == "ADCT_ERR_CANCELLED"]
        # the Python scheduler reports exactly what it withdrew; the native one
        # also accepts a request that was admitted meanwhile (it then runs)
        assert len(cancelled) == sum(flags) or server_cls is NativeServer
        assert len(cancelled) >= 1
        assert all(r.error is None for r in reqs if r.error != "ADCT_ERR_CANCELLED")
        assert all(r.result is None for r in cancelled)
        # a finished request cannot be cancelled any more
        assert not srv.cancel(reqs[0])
        # a decode of the newest encode that ran (older ones are evicted from
        # this small store) is still correct
        _, px_ref = oracle.roundtrip(big.numpy(), oracle.MODE_STEP, inputs.step_table(4))
        done_ok = [r for r in reqs if r.error is None][-1:]
        for r in done_ok:
            d = srv.decode(r.result)
            assert d.done.wait(30) and d.error is None
            assert np.array_equal(d.result.numpy(), px_ref)
        if server_cls is NativeServer:
            st = srv.stats
            assert st["cancelled"] == len(cancelled)
            assert sum(st["latency_hist"]) >= len(reqs)
    finally:
        srv.close()
