"""The multi-rank bench logic on CPU: two gloo ranks, no GPU.  Ranks shard the
images (disjoint seeds), never exchange data, and the whole-job rate is the
sum of units over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    d = bench.Dist(backend="gloo")
    d.barrier()
    units = 100.0 * (rank + 1)
    seconds = 1.0 + rank  # rank 1 is slower
    rate, t = bench.whole_job_rate(d, units, seconds)
    out[rank] = (rate, t, bench.shard_seed(rank, 256, 1702))
    d.close()


def test_two_ranks_reduce_like_the_benchmark():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (r0, t0, s0), (r1, t1, s1) = out[0], out[1]
    assert t0 == t1 == 2.0           # max over ranks
    assert r0 == r1 == 300.0 / 2.0   # all units over the slowest time
    assert s1 - s0 == 256             # disjoint image seeds


def test_single_process_needs_no_process_group():
    import bench
    d = bench.Dist()
    assert d.ws == 1 and d.pg is None
    assert bench.whole_job_rate(d, 10.0, 2.0) == (5.0, 2.0)
