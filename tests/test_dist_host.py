"""Multi-process host logic on CPU (gloo, world size 2): view sharding and the timing reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2012_03939_gb300 import scenes as S
from paper_2012_03939_gb300.dist import max_over_ranks, shard_views, sum_over_ranks, view_cost


def test_shard_views_partitions_and_balances():
    views = S.batched().views
    for world in (1, 2, 3, 8):
        parts = [shard_views(views, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(views)))
        loads = [sum(view_cost(views[i]) for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(view_cost(v) for v in views)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    views = S.batched().views
    mine = shard_views(views, rank, world)
    units = sum(view_cost(views[i]) for i in mine)
    ms = 10.0 + 5.0 * rank                      # the slower rank decides the job time
    t = max_over_ranks(ms)
    total = sum_over_ranks(units)
    dist.barrier()
    q.put((rank, mine, t, total))
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    views = S.batched().views
    assert sorted(out[0][1] + out[1][1]) == list(range(len(views)))
    assert out[0][2] == out[1][2] == 15.0
    assert out[0][3] == out[1][3] == sum(view_cost(v) for v in views)
