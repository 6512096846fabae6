#!/usr/bin/env python3
"""Benchmark of the 14-addition approximate DCT codec on GB300.

Default workload (one "step" = one pass of the whole integer path over one
batch): a uniform batch of 256 synthetic 1080x1920 uint8 images, round trip
(forward 2D transform, quantise, store int16 q, dequantise, inverse,
reconstruct) in ONE launch through the C ABI.  Steps cycle through the eight
quantiser settings: step tables Q_ij = 1 + floor(s (1 + i + j)) for s in
{1, 4, 16} and zonal retention r in {1, 6, 10, 16, 64}.

Prints one JSON line (rank 0).  Other workloads (--workload ragged | float |
serving) print their own lines.  --impl reference times the CPU oracle on the
host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "8x8 blocks/s and HBM GB/s (fraction of ~8 TB/s) for round trip; serving p50/p99"
BYTES_PER_BLOCK = 256  # 64 B pixels in, 128 B int16 q out, 64 B pixels out
N_IMG, H, W = 256, 1080, 1920
SETTINGS = [("step", 1), ("step", 4), ("step", 16), ("zonal", 1), ("zonal", 6), ("zonal", 10), ("zonal", 16),
            ("zonal", 64)]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["roundtrip"], default="roundtrip")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--images", type=int, default=N_IMG)
    return p.parse_args()


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self, backend="nccl"):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch
            import torch.distributed as dist
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = torch.device("cuda", self.local) if self.pg.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = torch.device("cuda", self.local) if self.pg.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- clocks
REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    """Polls NVML (read-only queries) for the SM clock and clock-event reasons
    while the timed region runs."""

    def __init__(self, device_index: int, period_s: float = 0.002):
        self.period = period_s
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self.ok = False
        self._stop = threading.Event()
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            uuid = None
            try:
                import torch
                uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            except Exception:
                pass
            rc = 1
            if uuid:
                rc = self.nvml.nvmlDeviceGetHandleByUUID(("GPU-" + uuid if not uuid.startswith("GPU-") else uuid)
                                                         .encode(), ctypes.byref(self.h))
            if rc != 0:
                rc = self.nvml.nvmlDeviceGetHandleByIndex_v2(device_index, ctypes.byref(self.h))
            if rc != 0:
                return
            try:
                self._reasons_fn = self.nvml.nvmlDeviceGetCurrentClocksEventReasons
            except AttributeError:
                self._reasons_fn = self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.ok = True
        except OSError:
            pass

    def _run(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if self._reasons_fn(self.h, ctypes.byref(rs)) == 0:
                self.reasons |= rs.value
            time.sleep(self.period)

    def start(self):
        if self.ok:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()

    def stop(self):
        if self.ok:
            self._stop.set()
            self._t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0}
        names = [n for b, n in REASONS.items() if self.reasons & b and n != "gpu_idle"]
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz, "reasons": names,
                "samples": len(self.samples)}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("adct_codec.cu", "adct_device.cuh"):
        with open(os.path.join(ROOT, "paper_1702_00817_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (otherwise None)."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel and parts[1] == cur:
            return float(parts[2])
    return None


def make_quants(make_quant, step_table, modes):
    from paper_1702_00817_gb300.codec import ADCT_Q_STEP, ADCT_Q_ZONAL
    out = []
    for kind, v in modes:
        if kind == "step":
            out.append(make_quant(ADCT_Q_STEP, step_table(v), 64))
        else:
            out.append(make_quant(ADCT_Q_ZONAL, None, v))
    return out


def cpu_oracle_blocks_per_s(planes, settings, target_cpu_s=10.0, cores=None):
    """Times the oracle (as it stands) on host threads over a bounded sample of
    planes of the workload; returns (blocks/s, cores, sample description)."""
    import numpy as np

    import oracle
    from paper_1702_00817_gb300 import inputs
    cores = cores or os.cpu_count() or 1
    h, w = planes[0].shape
    nb = (h // 8) * (w // 8)
    scratch = [np.empty(2 * nb * 64, np.int64) for _ in range(cores)]
    outs = [np.empty((h, w), np.uint8) for _ in range(cores)]

    def run(k, slot):
        kind, v = settings[k % len(settings)]
        if kind == "step":
            oracle.roundtrip_pixels_only(planes[k % len(planes)], oracle.MODE_STEP, inputs.step_table(v), 64,
                                         scratch[slot], outs[slot])
        else:
            oracle.roundtrip_pixels_only(planes[k % len(planes)], oracle.MODE_ZONAL, None, v, scratch[slot],
                                         outs[slot])

    t0 = time.perf_counter()
    run(0, 0)
    t1 = time.perf_counter() - t0
    count = max(cores, int(round(target_cpu_s / max(t1, 1e-6))))
    count = (count + cores - 1) // cores * cores
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda k: run(k, k % cores), range(count)))
    wall = time.perf_counter() - t0
    return count * nb / wall, cores, f"{count} planes of {h}x{w} ({count * nb} blocks), settings cycled, {cores} threads"


# ---------------------------------------------------------------- workloads
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    from paper_1702_00817_gb300 import inputs
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    planes = [inputs.synth_image(H, W, inputs.BASE_SEED + k)[0] for k in range(min(cores, N_IMG))]
    nb = (H // 8) * (W // 8)

    def step(i):
        def one(k):
            kind, v = SETTINGS[(i * cores + k) % len(SETTINGS)]
            if kind == "step":
                oracle.roundtrip(planes[k % len(planes)], oracle.MODE_STEP, inputs.step_table(v), 64)
            else:
                oracle.roundtrip(planes[k % len(planes)], oracle.MODE_ZONAL, None, v)
        with ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(one, range(cores)))

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    wall = time.perf_counter() - t0
    blocks = args.steps * cores * nb
    value = blocks / wall
    sample = f"per step {cores} planes of {H}x{W} (one per thread), settings cycled"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": f"uniform batch {N_IMG}x{H}x{W} u8 round trip (CPU oracle sample)",
                       "settings": [f"{k}{v}" for k, v in SETTINGS]},
            "cpu_baseline": {"value": value, "unit": "blocks/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_roundtrip(args):
    import numpy as np
    import torch

    from paper_1702_00817_gb300 import _build, inputs
    from paper_1702_00817_gb300.codec import Codec, Image, image_array, make_quant

    d = Dist()
    dev = torch.device("cuda", d.local)
    torch.cuda.set_device(dev)
    if d.rank == 0 or not _build.up_to_date():
        _build.build()
    d.barrier()
    n = args.images
    host = inputs.synth_batch(n, H, W, base_seed=inputs.BASE_SEED + d.rank * n)[:, 0]
    src = torch.from_numpy(host).to(dev)
    dst = torch.empty_like(src)
    coef = torch.empty((n, H // 8, W // 8, 8, 8), dtype=torch.int16, device=dev)
    codec = Codec(d.local)
    images = [Image(src[k], dst[k], coef[k:k + 1]) for k in range(n)]
    arr = image_array(images)
    quants = make_quants(make_quant, inputs.step_table, SETTINGS)
    stream = torch.cuda.current_stream(dev)
    sh = ctypes.c_void_p(stream.cuda_stream)
    lib, ctx = codec.lib, codec.ctx
    blocks = n * (H // 8) * (W // 8)

    def step(i):
        st = lib.adct_roundtrip(ctx, arr, n, ctypes.byref(quants[i % len(quants)]), sh)
        if st != 0:
            raise RuntimeError(lib.adct_last_error(ctx).decode())

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize()
    codec.kernel_time()  # reset counters
    codec.kernel_timing(True)
    sampler = ClockSampler(d.local)
    d.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.stop()
    d.barrier()
    codec.kernel_timing(False)
    kernel_ms, launches = codec.kernel_time()
    local_ms = e0.elapsed_time(e1)
    max_ms = d.max(local_ms)
    total_blocks = d.sum(blocks * args.steps)
    value = total_blocks / (max_ms / 1000.0)
    peak, peak_kind = measured_peaks()
    kern_avg_ms = kernel_ms / max(1, launches)
    achieved = blocks * BYTES_PER_BLOCK / (kern_avg_ms / 1000.0) / 1e9
    gbs = value * BYTES_PER_BLOCK / 1e9

    e2e = None
    if not args.no_e2e:
        hsrc = torch.from_numpy(host).pin_memory()
        hdst = torch.empty_like(hsrc).pin_memory()
        hcoef = torch.empty((n, H // 8, W // 8, 8, 8), dtype=torch.int16).pin_memory()
        himgs = [Image(hsrc[k], hdst[k], hcoef[k:k + 1]) for k in range(n)]
        harr = image_array(himgs)
        esteps = max(3, min(args.steps, 10))
        chunk = 64 << 20
        for i in range(2):
            st = lib.adct_roundtrip_host(ctx, harr, n, ctypes.byref(quants[i % len(quants)]), chunk)
            assert st == 0, lib.adct_last_error(ctx).decode()
        d.barrier()
        t0 = time.perf_counter()
        for i in range(esteps):
            st = lib.adct_roundtrip_host(ctx, harr, n, ctypes.byref(quants[i % len(quants)]), chunk)
            assert st == 0, lib.adct_last_error(ctx).decode()
        et = d.max(time.perf_counter() - t0)
        e2e = {"value": d.sum(blocks * esteps) / et, "unit": "blocks/s", "h2d_bytes_per_step": n * H * W,
               "d2h_bytes_per_step": n * H * W * 3, "steps": esteps, "api": "adct_roundtrip_host (pinned host buffers)"}

    cpu = None
    if not args.no_cpu and d.rank == 0 and d.ws == 1:
        bps, cores, sample = cpu_oracle_blocks_per_s([host[k] for k in range(min(8, n))], SETTINGS)
        cpu = {"value": bps, "unit": "blocks/s", "cores": cores, "kind": "oracle", "sample": sample}

    if d.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": d.ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"uniform batch {n}x{H}x{W} u8 round trip, one launch per step "
                                   f"(forward, quantise, int16 q out, inverse, u8 out)",
                       "images_per_gpu": n, "height": H, "width": W,
                       "settings": [f"{k}{v}" for k, v in SETTINGS],
                       "l2": f"inputs larger than L2 ({blocks * BYTES_PER_BLOCK / 1e9:.2f} GB touched per step)",
                       "parallelism": f"dp{d.ws} (images sharded per GPU, no collective)",
                       "launch": codec.get_launch()},
            "gbs": gbs, "hbm_frac": gbs / peak,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": f"{peak_kind} (copy, burst)", "kernel": "k_codec<RT_FULL>",
                         "traffic": recorded_traffic("k_codec_rt_full"),
                         "algorithmic_bytes_per_launch": blocks * BYTES_PER_BLOCK, "kernel_ms": kern_avg_ms},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": sampler.summary(),
        }
        print(json.dumps(line), flush=True)
    codec.close()
    d.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_roundtrip(args)


if __name__ == "__main__":
    sys.exit(main())
