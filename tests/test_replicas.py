"""Replica helpers over a 2-rank gloo process group on CPU (the multi-GPU path
shards whole extractions and only combines timings)."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2402_09481_gb300 import replicas


def test_shard_covers_disjointly():
    for count in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(count, world, r) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(count))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    share = replicas.shard(4096, world, rank)
    ms = 10.0 + 5.0 * rank                       # rank 1 is slower
    value, slowest = replicas.job_throughput(len(share), ms)
    dist.barrier()
    out.put((rank, len(share), value, slowest))
    dist.destroy_process_group()


def test_two_rank_gloo_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2048, 2048]
    for _, _, value, slowest in res:
        assert slowest == 15.0
        assert abs(value - 4096 / 0.015) < 1e-6
