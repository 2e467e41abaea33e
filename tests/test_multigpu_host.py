"""Multi-rank host logic on CPU: world size 2 over gloo (no GPU)."""
import os
import socket

import pytest

from paper_1205_5351_gb300 import multigpu


def test_shards_are_disjoint_and_cover():
    for total in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                seen += list(multigpu.shard(total, r, world))
            assert seen == list(range(total))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = multigpu.shard(10, rank, world)
        t = multigpu.max_over_ranks([1.0 + rank, 5.0 - rank], dist)
        n = multigpu.sum_over_ranks([float(len(mine))], dist)
        q.put((rank, t, n))
    finally:
        dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, n in out:
        assert t == [2.0, 5.0]          # max over ranks, element-wise
        assert n == [10.0]              # every problem counted once
