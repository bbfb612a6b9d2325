"""Host-side helpers for running on several GPUs, one process per GPU.

A single graph does not shard (every BFS level would need an exchange of
visited columns and matched rows), so one graph runs on one GPU and N GPUs
run N independent replicas.  A batch of independent graphs does shard: whole
graphs are dealt to ranks largest first (LPT), with no collective on the data
path -- only the timing reduction below.  A served request stream shards the
same way, by whole request: each arriving request goes to the rank with the
fewest edges so far, whose own server matches it.
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


# ------------------------------------------------------------------ served request streams
def assign_stream(edge_counts, world: int) -> np.ndarray:
    """Deals a request stream to ranks as it arrives: request i (in arrival
    order) goes to the rank with the fewest edges assigned so far (ties: the
    lowest rank).  Each rank computes the same deal from the same stream, so
    the ranks agree on it without exchanging a message; a request is served by
    exactly one rank."""
    heap = [(0, r) for r in range(world)]
    out = np.empty(len(edge_counts), dtype=np.int64)
    for i, e in enumerate(edge_counts):
        load, r = heapq.heappop(heap)
        out[i] = r
        heapq.heappush(heap, (load + int(e), r))
    return out


class StreamShard:
    """One rank's share of a served request stream.  `server` is this rank's
    matching server (an object with submit(n_rows, n_cols, col_ptr, row_idx)
    -> id, wait(id, timeout_s) -> dict with status, card and latency_ns, and
    release(id), as bmatch.Server); offer() submits request i only if the deal
    gives it to this rank, drain() waits for this rank's requests.  The ranks'
    results meet only after the stream, in gather_results()."""

    def __init__(self, server, rank: int, assignment):
        self.server = server
        self.rank = rank
        self.assignment = np.asarray(assignment)
        self.pending = []

    def mine(self, i: int) -> bool:
        return int(self.assignment[i]) == self.rank

    def offer(self, i: int, n_rows, n_cols, col_ptr, row_idx) -> bool:
        if not self.mine(i):
            return False
        self.pending.append((i, self.server.submit(n_rows, n_cols, col_ptr, row_idx)))
        return True

    def drain(self, timeout_s: float = 120.0):
        """[(request index, status, |M|, latency in ns)] of this rank's requests."""
        out = []
        for i, rid in self.pending:
            info = self.server.wait(rid, timeout_s)
            out.append((i, int(info["status"]), int(info["card"]), int(info["latency_ns"])))
            self.server.release(rid)
        self.pending = []
        return out


def gather_results(local):
    """Every rank's drained results, merged and sorted by request index
    (identity when torch.distributed is not initialised).  Host objects over
    the process group after the stream: not on the data path."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return sorted(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(local))
    return sorted(x for p in parts for x in p)
