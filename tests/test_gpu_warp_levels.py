"""The one-block-per-graph routine with its tree marks in shared memory
(batched kernel and serving workers, graphs of at most 61,440 columns, one
endpoint per root): BFS levels expanded by warps, columns of more than 256
edges expanded by the whole block, more such columns in one level than the
block sets aside (16), the cheap matching's row claims in shared memory and
graphs whose rows do not fit them, and the column limit of the bitmaps on
both sides.  Every graph's |M| equals Hopcroft-Karp's and its matching is
valid with a Koenig certificate; with the deterministic option (the same
warp walk with minimum claim rules) the matching and counters equal the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import bmatch, synth
from paper_1303_1379_gb300.synth import Graph

from helpers import assert_maximum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HUB_DEG = 256       # columns of more edges are expanded by the whole block
HUB_MAX = 16        # at most this many a level; the rest stay with their warp
SB_MAX_COLS = 61440  # bitmap capacity (columns for the search, rows for the cheap matching)

SB_VARIANTS = [dict(mode=0, bfs=1, wr_one_endpoint=1), dict(mode=1, bfs=1, wr_one_endpoint=1)]


def hub_graph(nr, nc, n_hubs, seed, base_max=4, hub_degs=None):
    """nc columns over nr rows: n_hubs of them (or those listed in hub_degs,
    column k getting hub_degs[k] rows) with 257..min(nr, 4000) distinct rows,
    the others 0..base_max rows; rows in random order inside a column."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, base_max + 1, size=nc)
    if hub_degs is not None:
        deg[:len(hub_degs)] = hub_degs
    else:
        hubs = rng.choice(nc, size=min(n_hubs, nc), replace=False)
        hi = min(nr, 4000)
        deg[hubs] = rng.integers(min(HUB_DEG + 1, hi), hi + 1, size=len(hubs))
    deg = np.minimum(deg, nr)
    lists = [rng.permutation(nr)[:d] if d > 64 else rng.choice(nr, size=d, replace=False) for d in deg]
    cp = np.zeros(nc + 1, np.int32)
    cp[1:] = np.cumsum(deg)
    ri = np.concatenate(lists).astype(np.int32) if cp[-1] else np.zeros(0, np.int32)
    return Graph(nr, nc, cp, ri, f"hub graph {nr}x{nc} seed {seed}")


def batch_of(graphs):
    nr = np.array([g.n_rows for g in graphs], np.int32)
    nc = np.array([g.n_cols for g in graphs], np.int32)
    ro = np.zeros(len(graphs) + 1, np.int64)
    np.cumsum(nr, out=ro[1:])
    co = np.zeros(len(graphs) + 1, np.int64)
    np.cumsum(nc, out=co[1:])
    eo = np.zeros(len(graphs) + 1, np.int64)
    np.cumsum([g.nnz for g in graphs], out=eo[1:])
    cp = np.concatenate([g.col_ptr for g in graphs]).astype(np.int32)
    ri = np.concatenate([g.row_idx for g in graphs]).astype(np.int32)
    return synth.Batch(nr, nc, ro, co, eo, cp, ri)


def match_batch(graphs, greedy, **options):
    b = batch_of(graphs)
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    rm = torch.full((max(R, 1),), -1, dtype=torch.int32, device="cuda")
    cm = torch.full((max(C, 1),), -1, dtype=torch.int32, device="cuda")
    card = torch.zeros(len(graphs), dtype=torch.int32, device="cuda")
    with bmatch.Batch.from_synth(b, **options) as bb:
        rc, _ = bb.match(rm, cm, greedy=greedy, card_out=card)
        status, _ = bb.graph_status()
    assert rc == 0 and np.all(status == 0), status
    rm, cm, card = rm[:R].cpu().numpy(), cm[:C].cpu().numpy(), card.cpu().numpy()
    for k, g in enumerate(graphs):
        want = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2]
        assert_maximum(g, rm[b.row_off[k]:b.row_off[k + 1]], cm[b.col_off[k]:b.col_off[k + 1]],
                       int(card[k]), want)


def hub_set(seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(20):
        nr = int(rng.integers(400, 6000))
        nc = max(1, int(nr * rng.uniform(0.8, 1.25)))
        out.append(hub_graph(nr, nc, int(rng.integers(0, 48)), seed=seed * 100 + i))
    return out


@pytest.mark.parametrize("greedy", [False, True])
@pytest.mark.parametrize("variant", SB_VARIANTS, ids=["APFB", "APsB"])
def test_hub_columns(variant, greedy):
    # from the empty matching every column with rows is a root of the first
    # level, so graphs with more than 16 hubs overflow the block's list there
    match_batch(hub_set(7), greedy, **variant)


def test_hub_degree_boundary_and_star():
    graphs = [
        # degrees exactly at and just above the threshold, and a full column (a star)
        hub_graph(3000, 2500, 0, seed=1, hub_degs=[HUB_DEG, HUB_DEG + 1, HUB_DEG - 1, 3000]),
        # every column a hub, more of them than the block takes in one level
        hub_graph(2000, 3 * HUB_MAX, 0, seed=2, base_max=0,
                  hub_degs=list(range(HUB_DEG + 1, HUB_DEG + 1 + 3 * HUB_MAX * 20, 20))),
        # one star column and nothing else
        hub_graph(1000, 1, 0, seed=3, hub_degs=[1000]),
        # a graph without edges, and one of a single edge
        Graph(5, 7, np.zeros(8, np.int32), np.zeros(0, np.int32), "no edges"),
        Graph(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), "one edge"),
    ]
    for greedy in (False, True):
        match_batch(graphs, greedy)


def test_rows_beyond_the_row_bitmap_and_column_limit():
    graphs = [
        synth.uniform_graph(SB_MAX_COLS + 8000, 30000, 6, seed=11),  # rows too many for the row claims
        synth.uniform_graph(SB_MAX_COLS, SB_MAX_COLS, 5, seed=12),   # both at the limit
        synth.uniform_graph(SB_MAX_COLS, SB_MAX_COLS + 1, 5, seed=13),  # one column over: level array
        hub_graph(SB_MAX_COLS + 100, 20000, 40, seed=14),
    ]
    for greedy in (False, True):
        match_batch(graphs, greedy)


def test_hub_requests_on_the_serving_workers():
    graphs = hub_set(9)[:12]
    assert all(g.nnz < (1 << 19) for g in graphs)  # below the large-request threshold: workers
    want = [oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2] for g in graphs]
    with bmatch.Server(keep_results=1, pool_bytes=1 << 30) as srv:
        for greedy in (False, True):
            ids = [srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, greedy=greedy) for g in graphs]
            for k, (g, rid) in enumerate(zip(graphs, ids)):
                info = srv.wait(rid)
                assert info["state"] == bmatch.BM_REQ_DONE and info["status"] == 0
                rm = np.empty(g.n_rows, np.int32)
                cm = np.empty(g.n_cols, np.int32)
                srv.fetch(rid, rm, cm)
                assert_maximum(g, rm, cm, info["card"], want[k])
                srv.release(rid)
        assert srv.stats()["exclusive_runs"] == 0


DET_STATS = ("phases", "levels", "endpoints", "inserted", "columns_expanded", "edges_scanned",
             "edges_to_matched", "alternate_steps")


@pytest.mark.parametrize("greedy", [False, True], ids=["empty", "rounds-greedy"])
def test_hub_columns_deterministic_same_as_the_oracle(greedy):
    # The deterministic option's block routine expands its levels by the same
    # warps and hands hubs to the whole block; its minima make the result the
    # oracle's, matching and counters alike, whatever the warps' order.
    graphs = hub_set(7)[:10] + [hub_graph(2000, 3 * HUB_MAX, 0, seed=2, base_max=0,
                                          hub_degs=list(range(HUB_DEG + 1, HUB_DEG + 1 + 3 * HUB_MAX * 20, 20)))]
    b = batch_of(graphs)
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    w_rm = np.full(R, -1, np.int32)
    w_cm = np.full(C, -1, np.int32)
    w_st = dict.fromkeys(DET_STATS, 0)
    for k, g in enumerate(graphs):
        rm0 = cm0 = None
        if greedy:
            rm0, cm0, _, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        rm, cm, _, st = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0)
        w_rm[b.row_off[k]:b.row_off[k + 1]] = rm
        w_cm[b.col_off[k]:b.col_off[k + 1]] = cm
        for key in DET_STATS:
            w_st[key] += st[key]
    rm = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    cm = torch.full((C,), -1, dtype=torch.int32, device="cuda")
    with bmatch.Batch.from_synth(b, deterministic=1) as bb:
        rc, st = bb.match(rm, cm, greedy=greedy)
        status, _ = bb.graph_status()
    assert rc == 0 and np.all(status == 0)
    np.testing.assert_array_equal(rm.cpu().numpy(), w_rm)
    np.testing.assert_array_equal(cm.cpu().numpy(), w_cm)
    assert {k: st[k] for k in DET_STATS} == w_st
