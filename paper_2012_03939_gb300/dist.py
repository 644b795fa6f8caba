"""Host-side helpers for running the path trace on several processes (one GPU each).

Views are independent given the scene, so work splits by view with no exchange
on the data path; an optimisation loop over several GPUs would add one
all-reduce of the vertex and parameter gradients per iteration. These helpers
cover the host side: a balanced view partition and the max-over-ranks timing
reduction used by the benchmark. They run on any torch.distributed backend
(``gloo`` on CPU in the tests, ``nccl`` on GPUs).
"""
from __future__ import annotations

from typing import List, Sequence

import torch


def view_cost(v) -> int:
    return int(v.width) * int(v.height) * max(int(v.spp), 1)


def shard_views(views: Sequence, rank: int, world: int) -> List[int]:
    """Indices of the views of ``rank``: longest-processing-time greedy on W*H*spp.

    Every view goes to exactly one rank; ties are broken by view index so all
    ranks compute the same partition without communicating.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    order = sorted(range(len(views)), key=lambda i: (-view_cost(views[i]), i))
    load = [0] * world
    owner = [0] * len(views)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += view_cost(views[i])
    return [i for i in range(len(views)) if owner[i] == rank]


def max_over_ranks(x: float, device="cpu") -> float:
    """Maximum of a per-rank float over the default process group (identity without one)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())
