"""The host side of multi-GPU runs with two ranks on CPU (gloo): shards of
independent units are disjoint and cover them, and the job's time and units
are the slowest rank's time and the sum of the ranks' units."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2505_22797_gb300 import multirank


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(multirank.shard(64, rank, world))
        multirank.barrier()
        t = multirank.max_over_ranks(1.0 + rank)          # rank 1 is slower
        u = multirank.sum_over_ranks(len(mine))
        rate = multirank.job_rate(len(mine), 1.0 + rank)
        out.put((rank, mine, t, u, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    units = [u for _, mine, _, _, _ in res for u in mine]
    assert sorted(units) == list(range(64))           # disjoint and covering
    for _, mine, t, u, rate in res:
        assert t == 2.0 and u == 64.0 and rate == 32.0


@pytest.mark.parametrize("n,world", [(64, 3), (5, 8), (0, 2), (7, 1)])
def test_shard_blocks(n, world):
    blocks = [multirank.shard(n, r, world) for r in range(world)]
    assert [u for b in blocks for u in b] == list(range(n))
    sizes = [len(b) for b in blocks]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_identity():
    assert multirank.max_over_ranks(3.5) == 3.5
    assert multirank.sum_over_ranks(2) == 2.0
    assert multirank.job_rate(10, 2.0) == 5.0
