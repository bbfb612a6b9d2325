"""Host-side helpers for running on several GPUs, one process per GPU.

A single graph does not shard (every BFS level would need an exchange of
visited columns and matched rows), so one graph runs on one GPU and N GPUs
run N independent replicas.  A batch of independent graphs does shard: whole
graphs are dealt to ranks largest first (LPT), with no collective on the data
path -- only the timing reduction below.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(sizes, world: int):
    """Deals items to `world` bins, largest first, each to the currently
    lightest bin (ties: lowest rank).  Returns one sorted index array per
    rank; every item appears exactly once."""
    sizes = np.asarray(sizes, dtype=np.int64)
    order = np.argsort(-sizes, kind="stable")
    heap = [(0, r) for r in range(world)]
    bins = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        bins[r].append(int(i))
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [np.array(sorted(b), dtype=np.int64) for b in bins]


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def sum_over_ranks(values, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()]
