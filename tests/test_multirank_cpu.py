"""The N > 1 host path on CPU ranks (gloo, world size 2): the largest-first
deal of a batch's graphs over ranks and the max / sum reductions that bench.py
uses to report whole-job throughput from per-rank timings."""
import os
import socket

import numpy as np
import pytest

from paper_1303_1379_gb300 import shard, synth

torch = pytest.importorskip("torch")


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = shard.lpt_partition(sizes, world)
    mine = parts[rank]
    load = float(np.asarray(sizes)[mine].sum())
    fake_ms = 10.0 + rank  # rank 1 is the slower one
    mx = shard.max_over_ranks([fake_ms, load])
    tot = shard.sum_over_ranks([len(mine), load])
    out.put((rank, mine.tolist(), mx, tot))
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_partition_is_exact_and_balanced():
    b = synth.batch_graphs(300, seed=3)
    sizes = np.diff(b.edge_off)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(sizes, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(sizes)))
        loads = [sizes[p].sum() for p in parts]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(loads) / world + sizes.max()


def test_two_gloo_ranks_agree_on_shards_and_reductions():
    import torch.multiprocessing as mp
    sizes = np.diff(synth.batch_graphs(64, seed=3).edge_off).tolist()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, mx0, t0), (r1, m1, mx1, t1) = res
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    assert mx0 == mx1 and mx0[0] == 11.0  # the slowest rank decides the time
    assert t0 == t1 and t0[0] == 64 and t0[1] == float(sum(sizes))
