"""Continuous-batching encode/decode server over the codec's C ABI.

Requests arrive at any time (Server.submit); a scheduler thread:
  1. takes new arrivals into a FIFO queue,
  2. retires launched batches whose completion events have fired (frees their
     temporary device memory, fills the results, stamps completion times),
  3. admits queued requests while the device-memory budget allows (evicting
     the oldest unreferenced entries of the on-device coefficient store when
     it must), and
  4. packs everything admitted in this pass into at most two ragged launches
     (one encode launch = forward + quantise with q kept on the device, one
     decode launch = dequantise + inverse) on the next of several CUDA
     streams, so batches admitted while others are still running overlap on
     the device.
Encode: pixels are copied from host memory, the quantised coefficients stay in
the store under a handle.  Decode: a stored handle is dequantised, inverted
and the pixels are copied back to host memory.  Results are bit-identical to a
request run alone (the kernels are per-block and deterministic).
"""
from __future__ import annotations

import collections
import itertools
import threading
import time
from dataclasses import dataclass, field

import torch

from .codec import ADCT_Q_STEP, Codec, Image, coef_per_block, make_quant


@dataclass
class Request:
    kind: str                       # "encode" or "decode"
    pixels: torch.Tensor | None = None   # encode: host uint8 [H, W] (pinned is fastest)
    handle: int | None = None       # decode: store handle
    t_arrival: float = 0.0
    t_sent: float = 0.0             # poisson_run: when the client handed it to submit (>= t_arrival)
    t_submitted: float = 0.0        # poisson_run: when submit returned
    t_admit: float = 0.0
    t_done: float = 0.0
    result: object = None           # encode: handle; decode: host uint8 [H, W]
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)
    # internal
    out_pixels: int = 0             # decode: pixels produced
    _need: int = 0
    _pinned: bool = False
    _dev: list = field(default_factory=list)
    _id: int = 0                    # NativeServer: the library's request id

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class CoefStore:
    """Quantised coefficients kept on the device, keyed by handle, oldest first."""

    def __init__(self):
        self.entries: collections.OrderedDict[int, dict] = collections.OrderedDict()
        self.bytes = 0

    def put(self, handle, coef, height, width):
        self.entries[handle] = {"coef": coef, "h": height, "w": width, "refs": 0}
        self.bytes += coef.numel() * 2

    def get(self, handle):
        return self.entries.get(handle)

    def evictable(self):
        return [h for h, e in self.entries.items() if e["refs"] == 0]

    def evict(self, handle) -> int:
        e = self.entries.pop(handle)
        nbytes = e["coef"].numel() * 2
        self.bytes -= nbytes
        return nbytes


class Server:
    def __init__(self, device: int = 0, budget_bytes: int = 4 << 30, streams: int = 4, quant=None,
                 codec: Codec | None = None, max_batch: int = 256):
        self.device = device
        self.dev = torch.device("cuda", device)
        self.codec = codec or Codec(device)
        self.budget = int(budget_bytes)
        self.quant = quant if quant is not None else make_quant(ADCT_Q_STEP, _default_table())
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self._stream_rr = itertools.cycle(range(streams))
        self.max_batch = max_batch
        self.store = CoefStore()
        self.in_flight_bytes = 0
        self._arrivals: collections.deque[Request] = collections.deque()
        self._queue: collections.deque[Request] = collections.deque()
        self._batches: list[tuple[torch.cuda.Event, list[Request]]] = []
        self._handles = itertools.count(1)
        self._lock = threading.Lock()
        self._wake = threading.Event()
        self._stop = False
        self.stats = {"launches": 0, "admitted": 0, "unknown_handle": 0, "oversized": 0, "evicted": 0,
                      "max_overlap": 0}
        self._thread = threading.Thread(target=self._loop, name="adct-server", daemon=True)
        self._thread.start()

    # -- client side -----------------------------------------------------
    def submit(self, req: Request) -> Request:
        if not req.t_arrival:
            req.t_arrival = time.perf_counter()
        with self._lock:
            if req.kind == "decode":
                # pin the handle while the request waits, so that admission of
                # other work cannot evict it in between
                e = self.store.get(req.handle)
                if e is not None:
                    e["refs"] += 1
                    req._pinned = True
            self._arrivals.append(req)
        self._wake.set()
        return req

    def encode(self, pixels: torch.Tensor) -> Request:
        return self.submit(Request("encode", pixels=pixels))

    def decode(self, handle: int) -> Request:
        return self.submit(Request("decode", handle=handle))

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that has not been admitted yet; it completes with
        error "ADCT_ERR_CANCELLED".  False when it is already running or done."""
        with self._lock:
            for q in (self._arrivals, self._queue):
                at = next((k for k, x in enumerate(q) if x is req), None)  # by identity
                if at is not None:
                    del q[at]
                    if req._pinned:
                        e = self.store.get(req.handle)
                        if e is not None:
                            e["refs"] -= 1
                        req._pinned = False
                    req.error = "ADCT_ERR_CANCELLED"
                    req.result = None
                    req.t_done = time.perf_counter()
                    self.stats["cancelled"] = self.stats.get("cancelled", 0) + 1
                    req.done.set()
                    return True
        return False

    def warm_host_buffers(self, shapes, count: int = 8) -> None:
        """Pre-fault pinned output buffers of the given [H, W] shapes so that
        decodes reuse them from torch's pinned-memory cache instead of calling
        the (slow, synchronising) pinned allocator on the request path."""
        bufs = [torch.empty(hw, dtype=torch.uint8, pin_memory=True) for hw in shapes for _ in range(count)]
        del bufs

    def drain(self, timeout: float = 60.0) -> None:
        t_end = time.perf_counter() + timeout
        while time.perf_counter() < t_end:
            with self._lock:
                busy = bool(self._arrivals or self._queue or self._batches)
            if not busy:
                return
            time.sleep(0.0005)
        raise TimeoutError("server did not drain")

    def close(self):
        self._stop = True
        self._wake.set()
        self._thread.join()

    # -- scheduler -------------------------------------------------------
    def _need_bytes(self, r: Request) -> int:
        if r.kind == "encode":
            H, W = r.pixels.shape
            return H * W + (H // 8) * (W // 8) * coef_per_block(self.quant) * 2  # pixels + int16 coefficients
        e = self.store.get(r.handle)
        return 0 if e is None else e["h"] * e["w"]  # output pixels

    def _retire(self):
        still = []
        for ev, reqs in self._batches:
            if ev.query():
                self._lock.acquire()
                now = time.perf_counter()
                for r in reqs:
                    if r.kind == "encode":
                        coef = r._dev[1]
                        H, W = r.pixels.shape
                        self.store.put(r.result, coef, H, W)  # the coefficients now count against the store
                        self.in_flight_bytes -= r._need
                    else:
                        e = self.store.get(r.handle)
                        e["refs"] -= 1
                        self.in_flight_bytes -= r._need
                    r._dev = []
                    r.t_done = now
                    r.done.set()
                self._lock.release()
            else:
                still.append((ev, reqs))
        self._batches = still

    def _used(self) -> int:
        return self.in_flight_bytes + self.store.bytes

    def _admit(self):
        with self._lock:
            return self._admit_locked()

    def _admit_locked(self):
        admitted = []
        while self._queue and len(admitted) < self.max_batch:
            r = self._queue[0]
            if r.kind == "decode" and (self.store.get(r.handle) is None):
                self._queue.popleft()
                r.error = "unknown handle"
                r.t_done = time.perf_counter()
                self.stats["unknown_handle"] += 1
                r.done.set()
                continue
            need = self._need_bytes(r)
            if need > self.budget:
                self._queue.popleft()
                r.error = "request larger than the device-memory budget"
                r.t_done = time.perf_counter()
                self.stats["oversized"] += 1
                r.done.set()
                continue
            while self._used() + need > self.budget:
                victims = [h for h in self.store.evictable() if not (r.kind == "decode" and h == r.handle)]
                if not victims:
                    break
                self.store.evict(victims[0])
                self.stats["evicted"] += 1
            if self._used() + need > self.budget:
                break  # wait for running batches to free memory
            self._queue.popleft()
            r._need = need
            r.t_admit = time.perf_counter()
            self.in_flight_bytes += need
            if r.kind == "decode" and not r._pinned:
                self.store.get(r.handle)["refs"] += 1
                r._pinned = True
            admitted.append(r)
        return admitted

    def _launch(self, reqs):
        enc = [r for r in reqs if r.kind == "encode"]
        dec = [r for r in reqs if r.kind == "decode"]
        for group, kind in ((enc, "encode"), (dec, "decode")):
            if not group:
                continue
            s = self.streams[next(self._stream_rr)]
            with torch.cuda.stream(s):
                imgs = []
                for r in group:
                    if kind == "encode":
                        H, W = r.pixels.shape
                        px = torch.empty((H, W), dtype=torch.uint8, device=self.dev)
                        px.copy_(r.pixels, non_blocking=True)
                        cpb = coef_per_block(self.quant)
                        shape = (1, H // 8, W // 8, 8, 8) if cpb == 64 else (1, H // 8, W // 8, cpb)
                        coef = torch.empty(shape, dtype=torch.int16, device=self.dev)
                        r._dev = [px, coef]
                        r.result = next(self._handles)
                        imgs.append(Image(px, None, coef))
                    else:
                        e = self.store.get(r.handle)
                        out = torch.empty((e["h"], e["w"]), dtype=torch.uint8, device=self.dev)
                        r._dev = [out]
                        imgs.append(Image(None, out, e["coef"]))
                if kind == "encode":
                    self.codec.roundtrip(imgs, self.quant, stream=s)
                else:
                    self.codec.inverse(imgs, self.quant, stream=s)
                    for r in group:
                        host = torch.empty(r._dev[0].shape, dtype=torch.uint8, pin_memory=True)
                        host.copy_(r._dev[0], non_blocking=True)
                        r.result = host
                        r.out_pixels = host.numel()
                ev = torch.cuda.Event()
                ev.record(s)
            self._batches.append((ev, group))
            self.stats["launches"] += 1
        self.stats["max_overlap"] = max(self.stats["max_overlap"], len(self._batches))

    def _loop(self):
        torch.cuda.set_device(self.dev)
        while not self._stop:
            with self._lock:
                while self._arrivals:
                    self._queue.append(self._arrivals.popleft())
            self._retire()
            admitted = self._admit()
            if admitted:
                self.stats["admitted"] += len(admitted)
                self._launch(admitted)
            if not admitted:
                if self._batches or self._queue:
                    time.sleep(0.00002)
                else:
                    self._wake.wait(0.001)
                    self._wake.clear()
        # finish outstanding work
        for ev, _ in self._batches:
            ev.synchronize()
        self._retire()


def _default_table():
    import numpy as np
    i = np.arange(8)[:, None]
    j = np.arange(8)[None, :]
    return (1 + np.floor(4 * (1 + i + j))).astype(np.uint16)


def poisson_run(server, rate: float, n_requests: int, sizes, images_by_size, seed: int = 0,
                warm_handles: int = 0, spin: bool = False):
    """Drive the server with a Poisson stream of n_requests (50/50 encode and
    decode; decodes pick a live handle).  Returns the finished requests; the
    pixels of finished decodes are released as the stream goes (only their
    timing is kept), as a client that consumed them would."""
    import numpy as np
    rng = np.random.default_rng(seed)
    live = []
    # warm-up encodes so decodes have handles
    warm = [server.encode(images_by_size[sizes[k % len(sizes)]][0]) for k in range(warm_handles)]
    for r in warm:
        r.done.wait(60)
        if r.error is None:
            live.append(r.result)
    gaps = rng.exponential(1.0 / rate, n_requests)
    kinds = rng.random(n_requests) < 0.5
    picks = rng.integers(0, len(sizes), n_requests)
    reqs = []
    pending_enc = []
    pending_dec = []
    t = time.perf_counter()
    for k in range(n_requests):
        t += gaps[k]
        wait = t - time.perf_counter()
        if spin:
            # the native scheduler needs no interpreter lock: spin for the last 200 us
            if wait > 2e-4:
                time.sleep(wait - 2e-4)
            while time.perf_counter() < t:
                pass
        elif wait > 0:
            time.sleep(wait)  # no busy wait: the arrival time stays t, lateness counts as latency
        # handles of finished encodes become decodable; decodes pick among the most recent
        if k % 8 == 0:
            done = [x for x in pending_enc if x.done.is_set()]
            pending_enc = [x for x in pending_enc if not x.done.is_set()]
            live.extend(x.result for x in done if x.error is None)
            live = live[-64:]
            still = []
            for x in pending_dec:
                if x.done.is_set():
                    x.result = None
                else:
                    still.append(x)
            pending_dec = still
        if kinds[k] or not live:
            imgs = images_by_size[sizes[picks[k]]]
            r = Request("encode", pixels=imgs[k % len(imgs)], t_arrival=t)
            pending_enc.append(r)
        else:
            r = Request("decode", handle=live[int(rng.integers(0, len(live)))], t_arrival=t)
            pending_dec.append(r)
        r.t_sent = time.perf_counter()
        server.submit(r)
        r.t_submitted = time.perf_counter()
        reqs.append(r)
    for r in reqs:
        r.done.wait(120)
        if r.kind == "decode":
            r.result = None
    return reqs


class NativeServer:
    """The same service run by the library's C++ scheduler (adct_server_*):
    admission, arena allocation, the coefficient store, batching, launches and
    completion tracking all happen on a native thread; this class only submits
    requests and turns completions into finished Request objects (a polling
    thread).  Interface compatible with Server for the client helpers."""

    def __init__(self, device: int = 0, budget_bytes: int = 4 << 30, streams: int = 4, quant=None,
                 max_batch: int = 256):
        import ctypes

        from . import _native as N
        self._N = N
        self._ct = ctypes
        self.lib = N.load()
        cfg = N.adct_server_config()
        cfg.budget_bytes = int(budget_bytes)
        cfg.streams = int(streams)
        cfg.max_batch = int(max_batch)
        cfg.quant = quant if quant is not None else make_quant(ADCT_Q_STEP, _default_table())
        h = ctypes.c_void_p()
        N.check(self.lib.adct_server_create(ctypes.byref(h), int(device), ctypes.byref(cfg)), None,
                "adct_server_create")
        self._srv = h
        self._lock = threading.Lock()
        self._pending: dict[int, Request] = {}
        self._shapes: dict[int, tuple[int, int]] = {}
        self._stop = False
        self._thread = threading.Thread(target=self._poll_loop, name="adct-native-poll", daemon=True)
        self._thread.start()

    def clock(self) -> float:
        return self.lib.adct_server_clock()

    # -- client side -----------------------------------------------------
    def submit(self, req: Request) -> Request:
        ct, N = self._ct, self._N
        rid = ct.c_uint64(0)
        t_sub = req.t_arrival or 0.0
        with self._lock:
            if req.kind == "encode":
                px = req.pixels
                if px.is_cuda or px.dtype != torch.uint8 or px.dim() != 2 or px.stride(1) != 1:
                    raise ValueError("NativeServer encodes host uint8 [H, W] tensors with unit column stride")
                H, W = px.shape
                st = self.lib.adct_server_encode(self._srv, px.data_ptr(), W, H, px.stride(0), t_sub, ct.byref(rid))
            else:
                shape = self._shapes.get(req.handle)
                if shape is None:
                    st = N.ADCT_ERR_INVALID_ARG
                else:
                    out = torch.empty(shape, dtype=torch.uint8, pin_memory=True)
                    req.result = out
                    w, h = ct.c_int32(0), ct.c_int32(0)
                    st = self.lib.adct_server_decode(self._srv, int(req.handle), out.data_ptr(), out.stride(0),
                                                     t_sub, ct.byref(rid), ct.byref(w), ct.byref(h))
                    req.out_pixels = out.numel()
            if st != N.ADCT_OK:
                req.error = "unknown handle" if req.kind == "decode" else self.lib.adct_status_string(st).decode()
                req.result = None
                req.t_done = time.perf_counter()
                if not req.t_arrival:
                    req.t_arrival = req.t_done
                req.done.set()
                return req
            self._pending[rid.value] = req
            req._id = rid.value
        return req

    def encode(self, pixels: torch.Tensor) -> Request:
        return self.submit(Request("encode", pixels=pixels))

    def decode(self, handle: int) -> Request:
        return self.submit(Request("decode", handle=handle))

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that has not been admitted yet (adct_server_cancel);
        it completes with error "ADCT_ERR_CANCELLED" if it had not run."""
        return req._id != 0 and self.lib.adct_server_cancel(self._srv, req._id) == self._N.ADCT_OK

    def _poll_loop(self):
        ct, N = self._ct, self._N
        buf = (N.adct_completion * 64)()
        while not self._stop:
            n = self.lib.adct_server_poll(self._srv, buf, 64, 1000)
            for k in range(n):
                c = buf[k]
                with self._lock:
                    r = self._pending.pop(c.request_id, None)
                    if r is None:
                        continue
                    if c.status == N.ADCT_OK and c.kind == 0:
                        self._shapes[c.handle] = tuple(r.pixels.shape)
                r.t_arrival = r.t_arrival or c.t_submit
                r.t_admit, r.t_done = c.t_admit, c.t_done
                if c.status != N.ADCT_OK:
                    r.error = self.lib.adct_status_string(c.status).decode()
                    if r.kind == "decode":
                        r.result = None
                elif r.kind == "encode":
                    r.result = c.handle
                r.done.set()

    @property
    def stats(self) -> dict:
        st = self._N.adct_server_stats_t()
        self.lib.adct_server_stats(self._srv, self._ct.byref(st))
        out = {f: getattr(st, f) for f, _ in st._fields_ if f not in ("reserved", "latency_hist")}
        out["latency_hist"] = list(st.latency_hist)
        return out

    def drain(self, timeout: float = 60.0) -> None:
        t_end = time.perf_counter() + timeout
        while time.perf_counter() < t_end:
            with self._lock:
                if not self._pending:
                    return
            time.sleep(0.0005)
        raise TimeoutError("server did not drain")

    def close(self):
        if self._srv:
            self.drain()
            self._stop = True
            self._thread.join()
            self.lib.adct_server_destroy(self._srv)
            self._srv = None
