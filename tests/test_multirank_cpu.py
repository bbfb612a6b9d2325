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


# ------------------------------------------------------------------ served streams
class OracleServer:
    """Stands in for one rank's GPU server on the CPU: a request's |M| is the
    oracle's Hopcroft-Karp value, its id the submission order."""

    def __init__(self):
        self.reqs = {}

    def submit(self, n_rows, n_cols, col_ptr, row_idx):
        import oracle
        rid = len(self.reqs)
        self.reqs[rid] = oracle.hopcroft_karp(n_rows, n_cols, col_ptr, row_idx)[2]
        return rid

    def wait(self, rid, timeout_s):
        return {"status": 0, "card": self.reqs[rid], "latency_ns": 1000 + rid}

    def release(self, rid):
        self.reqs.pop(rid)


def stream_graphs(n=40):
    rng = np.random.default_rng(7)
    out = []
    for i in range(n):
        nr = int(rng.integers(50, 600))
        nc = int(rng.integers(50, 600))
        if i % 2:
            out.append(synth.uniform_graph(nr, nc, int(rng.integers(1, 9)), seed=100 + i))
        else:
            out.append(synth.rmat_graph(int(np.ceil(np.log2(max(nr, nc)))), 4 * max(nr, nc), seed=100 + i,
                                        n=max(nr, nc)))
    return out


def _serve_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    graphs = stream_graphs()
    deal = shard.assign_stream([g.nnz for g in graphs], world)
    sh = shard.StreamShard(OracleServer(), rank, deal)
    offered = [i for i, g in enumerate(graphs) if sh.offer(i, g.n_rows, g.n_cols, g.col_ptr, g.row_idx)]
    local = sh.drain()
    merged = shard.gather_results(local)
    out.put((rank, offered, [x[0] for x in local], merged))
    dist.barrier()
    dist.destroy_process_group()


def test_stream_deal_is_online_least_loaded():
    edges = [5, 1, 1, 1, 9, 2, 2, 2, 2]
    deal = shard.assign_stream(edges, 2)
    # loads after each request: (5,0) (5,1) (5,2) (5,3) (5,12) (7,12) (9,12) (11,12) (13,12)
    assert deal.tolist() == [0, 1, 1, 1, 1, 0, 0, 0, 0]
    loads = [sum(e for e, r in zip(edges, deal) if r == k) for k in range(2)]
    assert abs(loads[0] - loads[1]) <= max(edges)
    big = np.diff(synth.batch_graphs(200, seed=3).edge_off)
    for world in (1, 3, 8):
        d = shard.assign_stream(big, world)
        assert set(d.tolist()) <= set(range(world))
        loads = np.bincount(d, weights=big, minlength=world)
        assert loads.max() - loads.min() <= big.max()


def test_two_gloo_ranks_serve_a_stream_exactly_once():
    """Each request of the stream is served by exactly one of two CPU ranks,
    and the gathered |M| per request equals the single-rank result."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_serve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, off0, loc0, merged0), (_, off1, loc1, merged1) = res
    graphs = stream_graphs()
    n = len(graphs)
    assert sorted(off0 + off1) == list(range(n)) and not set(off0) & set(off1)
    assert off0 == loc0 and off1 == loc1 and off0 and off1
    assert merged0 == merged1 and [x[0] for x in merged0] == list(range(n))
    single = shard.StreamShard(OracleServer(), 0, shard.assign_stream([g.nnz for g in graphs], 1))
    for i, g in enumerate(graphs):
        assert single.offer(i, g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    alone = shard.gather_results(single.drain())
    assert [(i, s, c) for i, s, c, _ in merged0] == [(i, s, c) for i, s, c, _ in alone]
