"""The multi-rank bench logic on CPU: two gloo ranks, no GPU.  Ranks shard the
images (disjoint seeds), never exchange data, and the whole-job rate is the
sum of units over the slowest rank's time."""
import os
import socket

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


def _plan_worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    from paper_1702_00817_gb300 import inputs
    from paper_1702_00817_gb300.codec import shard_plan
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [(3, h, w) for h, w in inputs.ragged_sizes(300, seed=17)]
    mine, mx = shard_plan(sizes, world, rank)  # computed locally, no exchange
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)  # only to check the plans, not part of the data path
    out[rank] = (everyone, mx)
    dist.destroy_process_group()


def test_ragged_batch_shards_without_exchange():
    """Two gloo ranks each compute their share of one ragged batch; together
    the shares cover every image once and are balanced by block count."""
    from paper_1702_00817_gb300 import inputs
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_plan_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    plans0, mx0 = out[0]
    plans1, mx1 = out[1]
    assert plans0 == plans1 and mx0 == mx1  # both ranks hold the same plan
    sizes = inputs.ragged_sizes(300, seed=17)
    blocks = [3 * (h // 8) * (w // 8) for h, w in sizes]
    assert sorted(plans0[0] + plans0[1]) == list(range(300))
    loads = [sum(blocks[i] for i in p) for p in plans0]
    assert max(loads) == mx0
    assert max(loads) - min(loads) <= max(blocks)  # greedy largest-first bound
