"""The multi-GPU path is replicas only (events are independent): check, with two gloo ranks
on the CPU, that the benchmark's event sharding is disjoint and its timing reduction takes the
slowest rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = bench.shard_plan(rank, world, 4, 100)
    got = [None] * world
    dist.all_gather_object(got, plan)
    t = bench.max_over_ranks(1.0 + rank, world, "cpu")
    if rank == 0:
        out.put((got, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_disjoint_and_time_is_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [s for plan in got for s, _ in plan]
    ids = [i for plan in got for _, i in plan]
    assert len(set(seeds)) == len(seeds) == 8
    assert len(set(ids)) == len(ids) == 8
    assert t == 2.0
