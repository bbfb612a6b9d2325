"""Parity of the CUDA path (through the C-ABI) with the oracle.

The bar: |M| bit-exact against Hopcroft-Karp, the returned matching valid and
carrying a Koenig certificate of maximality; for a full GPUBFS pass the level
of every column and the set of reached unmatched rows equal the oracle's
alternating BFS exactly (those are unique); where several answers are correct
(which maximum matching, GPUBFS-WR trees) the test checks validity instead.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import bmatch, synth

from helpers import (VARIANTS, assert_maximum, csr_from_edges, gpu_match, oracle_max, to_dev,
                     vname)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_workloads():
    out = {}
    with open(os.path.join(GOLDEN, "workloads.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                out[line[0]] = {k: int(v) if v.lstrip("-").isdigit() else v
                                for k, v in (kv.split("=") for kv in line[1:])}
    return out


@pytest.fixture(scope="module")
def c1():
    return synth.workload("uniform10k")


@pytest.mark.parametrize("variant", VARIANTS, ids=vname)
def test_variants_on_uniform10k(c1, variant):
    want = golden_workloads()["uniform10k"]["max"]
    rm, cm, card, st = gpu_match(c1, **variant)
    assert_maximum(c1, rm, cm, card, want)
    assert st["initial_card"] == 0 and st["final_card"] == want
    assert st["phases"] >= 2 and st["levels"] >= st["phases"] - 1


@pytest.mark.parametrize("variant", VARIANTS[:6], ids=vname)
def test_variants_from_greedy_ragged(variant):
    # ragged sizes: nothing is a multiple of 32 or of a block
    g = synth.uniform_graph(7919, 8111, 5, seed=21)
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    rm, cm, card, st = gpu_match(g, (rm0, cm0), **variant)
    assert_maximum(g, rm, cm, card, oracle_max(g))
    assert st["initial_card"] == int((cm0 >= 0).sum())


@pytest.mark.parametrize("seed", range(12))
def test_random_rectangular_small(seed):
    rng = np.random.default_rng(100 + seed)
    nr, nc = int(rng.integers(1, 400)), int(rng.integers(1, 400))
    g = synth.uniform_graph(nr, nc, int(rng.integers(1, 12)), seed=seed)
    v = VARIANTS[seed % len(VARIANTS)]
    rm, cm, card, _ = gpu_match(g, **v)
    assert_maximum(g, rm, cm, card, oracle_max(g))


def bfs_gpu(g, init, **options):
    cp, ri = to_dev(g)
    m = bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, **options)
    try:
        m.set_matching(torch.from_numpy(init[0]).cuda(), torch.from_numpy(init[1]).cuda())
        lv = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
        rt = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
        pd = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        ep = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        n = m.bfs(lv, rt, pd, ep)
        after_r = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        after_c = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
        m.get_matching(after_r, after_c)
        assert np.array_equal(after_r.cpu().numpy(), init[0])  # BFS leaves the matching as installed
        assert np.array_equal(after_c.cpu().numpy(), init[1])
        return lv.cpu().numpy(), rt.cpu().numpy(), pd.cpu().numpy(), ep[:n].cpu().numpy()
    finally:
        m.close()


@pytest.mark.parametrize("gname", ["uniform", "rmat", "stencil"])
def test_gpubfs_levels_equal_alternating_bfs(gname):
    """A full GPUBFS pass (APFB, Algorithm 2) assigns every column its
    alternating BFS distance from the free columns, offset by L0 = 2, and
    reaches exactly the unmatched rows adjacent to reached columns."""
    g = {"uniform": lambda: synth.uniform_graph(20011, 19993, 6, seed=4),
         "rmat": lambda: synth.rmat_graph(15, 200000, seed=5),
         "stencil": lambda: synth.stencil_graph(150, 2250, 0.05, seed=6)}[gname]()
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    want_level, want_reached = oracle.bfs_levels(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0, L0=2)
    level, root, pred, ends = bfs_gpu(g, (rm0, cm0), mode=0, bfs=0)
    assert np.array_equal(level, want_level)
    assert sorted(ends.tolist()) == np.flatnonzero(want_reached).tolist()
    assert np.all(root == -1)
    # every reached matched column was entered through its own row from a column one level up
    reached = np.flatnonzero(level > 2)
    r = cm0[reached]
    p = pred[r]
    assert np.all(level[p] == level[reached] - 1)
    for c_prev, row in zip(p[:500], r[:500]):
        assert row in g.row_idx[g.col_ptr[c_prev]:g.col_ptr[c_prev + 1]]


def level_widths(level):
    """Columns per BFS level (the frontier each level expands), level L0 = 2 first."""
    vals, counts = np.unique(level[level >= 2], return_counts=True)
    return dict(zip(vals.tolist(), counts.tolist()))


@pytest.mark.parametrize("gname", ["uniform1M", "rmat21"])
@pytest.mark.parametrize("driver", [0, 1], ids=["persistent", "host"])
def test_gpubfs_levels_equal_alternating_bfs_wide(gname, driver):
    """The exact level pin on frontiers far wider than the grid: the
    persistent kernel expands a level of at most 32,768 columns through the
    row stamps, a level of up to one tile per block (grid x 512 columns) by
    block index with a level CAS, and a wider level in guided ranges from a
    position counter; the host loop's per-level launches take fixed tiles from
    a counter.  Every path must give each column its alternating BFS distance
    and claim exactly the reachable free rows (Algorithm 2, APFB)."""
    g = {"uniform1M": lambda: synth.uniform_graph(1_000_000, 1_000_000, 4, seed=4),
         "rmat21": lambda: synth.workload("rmat21")}[gname]()
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    want_level, want_reached = oracle.bfs_levels(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0, L0=2)
    # the frontier of level L0 is the free columns that have rows
    widths = level_widths(want_level)
    widths[2] = int(((cm0 < 0) & (np.diff(g.col_ptr) > 0)).sum())
    level, root, pred, ends = bfs_gpu(g, (rm0, cm0), mode=0, bfs=0, driver=driver)
    assert np.array_equal(level, want_level)
    assert np.array_equal(np.sort(ends), np.flatnonzero(want_reached))
    assert np.all(root == -1)
    reached = np.flatnonzero(level > 2)
    assert np.all(level[pred[cm0[reached]]] == level[reached] - 1)
    if driver == 0:
        # the three claim paths were all taken (widths from the oracle)
        stats = gpu_match(g, (rm0, cm0), mode=0, bfs=0)[3]
        one_tile_per_block = stats["grid"] * stats["block"]
        w = list(widths.values())
        assert any(x > one_tile_per_block for x in w), (widths, one_tile_per_block)
        assert any(x <= 32768 for x in w)
        if gname == "uniform1M":
            assert any(32768 < x <= one_tile_per_block for x in w), (widths, one_tile_per_block)


@pytest.mark.parametrize("gname", ["uniform", "rmat", "stencil"])
@pytest.mark.parametrize("driver", [0, 1], ids=["persistent", "host"])
def test_apsb_gpubfs_stops_after_the_first_level_with_an_endpoint(gname, driver):
    """APsB (Algorithm 1's break): the search expands levels L0, L0 + 1, ...
    until the first level k* whose columns reach an unmatched row, completes
    that level and stops.  So exactly the columns at alternating distance
    <= k* + 1 - L0 are reached, at their distance, and the endpoints are the
    unmatched rows adjacent to the columns of level k* (reading 11)."""
    g = {"uniform": lambda: synth.uniform_graph(20011, 19993, 6, seed=4),
         "rmat": lambda: synth.rmat_graph(15, 200000, seed=5),
         "stencil": lambda: synth.stencil_graph(150, 2250, 0.05, seed=6)}[gname]()
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    full, _ = oracle.bfs_levels(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0, L0=2)
    deg = np.diff(g.col_ptr)
    col_of_edge = np.repeat(np.arange(g.n_cols), deg)
    free_edge = rm0[g.row_idx] == -1
    # the first frontier level that touches an unmatched row
    touching = np.unique(full[col_of_edge[free_edge]])
    kstar = int(touching[touching >= 2].min())
    want_level = np.where((full >= 2) & (full <= kstar + 1), full, 1)
    want_ends = np.unique(g.row_idx[free_edge & (full[col_of_edge] == kstar)])
    level, root, pred, ends = bfs_gpu(g, (rm0, cm0), mode=1, bfs=0, driver=driver)
    assert np.array_equal(level, want_level)
    assert np.array_equal(np.sort(ends), want_ends)


@pytest.mark.parametrize("one_ep", [1, 0])
def test_gpubfs_wr_trees_are_valid(one_ep):
    """GPUBFS-WR trees depend on timing; check what must hold: levels never
    beat the true distance, every reached column hangs off a column of the same
    root one level up, and (one endpoint per root) each served root stores
    -(its endpoint row)."""
    g = synth.uniform_graph(30011, 30011, 4, seed=8)
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    dist, _ = oracle.bfs_levels(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0, L0=2)
    level, root, pred, ends = bfs_gpu(g, (rm0, cm0), mode=0, bfs=1, wr_one_endpoint=one_ep)
    free_cols = np.flatnonzero(cm0 < 0)
    assert np.all(root[free_cols] == free_cols)
    inner = np.flatnonzero(level > 2)
    assert np.all(level[inner] >= dist[inner]) and np.all(dist[inner] > 1)
    eff = level.copy()
    eff[free_cols] = 2  # a served root's slot holds its endpoint mark, its level is L0
    p = pred[cm0[inner]]
    assert np.all(eff[p] == level[inner] - 1)
    assert np.all(root[inner] == root[p])
    assert len(ends) > 0 and np.all(rm0[ends] == -1)
    ends_root = root[pred[ends]]
    if one_ep:
        assert len(set(ends_root.tolist())) == len(ends)  # one endpoint per root
        assert np.all(level[ends_root] == -ends)
    else:
        assert np.all(level[ends_root] == 0)


def test_fig1_race_example():
    d = {"edge": [], "match": []}
    with open(os.path.join(GOLDEN, "fig1_race.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                v = [int(x) for x in v]
                if k in ("edge", "match"):
                    d[k].append(tuple(v))
                else:
                    d[k] = v if len(v) != 1 else v[0]
    g = csr_from_edges(d["n_rows"], d["n_cols"], d["edge"])
    rm0 = np.full(g.n_rows, -1, np.int32)
    cm0 = np.full(g.n_cols, -1, np.int32)
    for r, c in d["match"]:
        rm0[r], cm0[c] = c, r
    level, _, _, ends = bfs_gpu(g, (rm0, cm0), mode=0, bfs=0)
    assert level.tolist() == d["expect_level"]
    assert sorted(ends.tolist()) == d["expect_reached_free_rows"]
    for v in VARIANTS:
        rm, cm, card, _ = gpu_match(g, (rm0, cm0), **v)
        assert_maximum(g, rm, cm, card, d["expect_max"])


def test_edge_cases():
    cases = [
        csr_from_edges(5, 4, []),                                   # no edges
        csr_from_edges(0, 3, []),                                   # no rows
        csr_from_edges(3, 0, []),                                   # no columns
        csr_from_edges(1, 1, [(0, 0)]),
        csr_from_edges(40, 70, [(r, c) for r in range(40) for c in range(70)]),   # K_{40,70}
        csr_from_edges(3000, 1, [(r, 0) for r in range(3000)]),     # one hub column
        csr_from_edges(1, 3000, [(0, c) for c in range(3000)]),     # every column on one row
        csr_from_edges(6, 3, [(5, 0), (1, 0), (5, 0), (1, 1), (3, 1), (1, 1), (0, 2)], keep_order=True),
    ]
    for g in cases:
        want = oracle_max(g) if g.n_rows and g.n_cols else 0
        for v in (VARIANTS[0], VARIANTS[2], VARIANTS[6]):
            rm, cm, card, _ = gpu_match(g, **v)
            assert card == want
            if g.n_rows and g.n_cols:
                assert_maximum(g, rm, cm, card, want)


def broom(n_handles, n_bristles, depth):
    """n_handles free columns share one chain of `depth` matched (row, column)
    pairs that ends in a column adjacent to n_bristles free rows: every search
    tree reaches the same bristles through the same suffix (the Fig. 1 pattern
    scaled up)."""
    edges, match = [], []
    nr = depth + n_bristles
    nc = n_handles + depth
    for h in range(n_handles):
        edges.append((0, h))                      # handle -> first chain row
    for k in range(depth):
        col = n_handles + k
        edges.append((k, col))                    # chain row k matched to chain column k
        match.append((k, col))
        if k + 1 < depth:
            edges.append((k + 1, col))
    last = n_handles + depth - 1
    for b in range(n_bristles):
        edges.append((depth + b, last))
    return csr_from_edges(nr, nc, edges), match


@pytest.mark.parametrize("block", [32, 96, 256, 512, 1024])
def test_race_stress_broom(block):
    g, match = broom(n_handles=700, n_bristles=900, depth=40)
    rm0 = np.full(g.n_rows, -1, np.int32)
    cm0 = np.full(g.n_cols, -1, np.int32)
    for r, c in match:
        rm0[r], cm0[c] = c, r
    want = oracle_max(g)
    for v in VARIANTS:
        for _ in range(3):
            rm, cm, card, _ = gpu_match(g, (rm0, cm0), block_size=block, **v)
            assert_maximum(g, rm, cm, card, want)


def test_gpu_greedy_is_maximal():
    g = synth.uniform_graph(50000, 52000, 6, seed=12)
    cp, ri = to_dev(g)
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri) as m:
        card = m.greedy()
        rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
        m.get_matching(rm, cm)
        rm, cm = rm.cpu().numpy(), cm.cpu().numpy()
    assert oracle.validate(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm) == (0, card)
    free_cols = np.flatnonzero(cm < 0)
    for c in free_cols:  # maximal: every row of an unmatched column is matched
        assert np.all(rm[g.row_idx[g.col_ptr[c]:g.col_ptr[c + 1]]] >= 0)


def heavy_mix_graph():
    """Columns in all three passes of the cheap matching: 40 heavy columns of
    2,500-6,000 rows over the first rows, 600 medium ones of 40-1,500 rows,
    and 20,000 light ones of 1-8 rows, all competing for the same low rows
    first (sorted lists), in shuffled column order."""
    rng = np.random.default_rng(31)
    nr = 30000
    cols = []
    for _ in range(40):
        cols.append(np.sort(rng.choice(8000, int(rng.integers(2500, 6001)), replace=False)))
    for _ in range(600):
        cols.append(np.sort(rng.choice(12000, int(rng.integers(40, 1501)), replace=False)))
    for _ in range(20000):
        cols.append(np.sort(rng.choice(nr, int(rng.integers(1, 9)), replace=False)))
    order = rng.permutation(len(cols))
    cols = [cols[k] for k in order]
    col_ptr = np.zeros(len(cols) + 1, np.int32)
    col_ptr[1:] = np.cumsum([len(c) for c in cols])
    return synth.Graph(nr, len(cols), col_ptr, np.concatenate(cols).astype(np.int32), "heavy-mix")


def assert_maximal_extension(g, rm, cm, card, rm0=None, cm0=None):
    assert oracle.validate(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm) == (0, card)
    deg = np.diff(g.col_ptr)
    free_cols = np.repeat(cm < 0, deg)  # per edge: is its column unmatched?
    assert np.all(rm[g.row_idx[free_cols]] >= 0)  # maximal: no edge joins two free vertices
    if rm0 is not None:  # the installed pairs stay
        kept = cm0 >= 0
        assert np.array_equal(cm[kept], cm0[kept]) and np.array_equal(rm[rm0 >= 0], rm0[rm0 >= 0])


@pytest.mark.parametrize("gname", ["heavy-mix", "rmat18"])
def test_gpu_greedy_passes_are_maximal(gname):
    """The three passes of the cheap matching (a thread, a warp, a block per
    column by degree) give a valid, maximal matching on graphs with columns
    of every class, from the empty matching and on top of an installed one."""
    g = heavy_mix_graph() if gname == "heavy-mix" else synth.rmat_graph(18, 1 << 22, seed=3)
    deg = np.diff(g.col_ptr)
    assert (deg > 2048).sum() >= 10 and ((deg > 32) & (deg <= 2048)).sum() >= 100 and (deg <= 32).sum() > 1000
    cp, ri = to_dev(g)
    rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
    cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri) as m:
        card = m.greedy()
        m.get_matching(rm, cm)
        assert_maximal_extension(g, rm.cpu().numpy(), cm.cpu().numpy(), card)
        # on top of a partial matching: every third pair of the oracle's greedy start
        rg, cg, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        rm0, cm0 = oracle.empty_matching(g.n_rows, g.n_cols)
        for c in np.flatnonzero(cg >= 0)[::3]:
            rm0[cg[c]], cm0[c] = c, cg[c]
        m.set_matching(torch.from_numpy(rm0).cuda(), torch.from_numpy(cm0).cuda())
        card = m.greedy()
        m.get_matching(rm, cm)
        assert_maximal_extension(g, rm.cpu().numpy(), cm.cpu().numpy(), card, rm0, cm0)
        res = m.match()
    assert res.card == oracle_max(g)


def test_match_from_equals_set_matching_then_match():
    """bm_match_from (install + Algorithm 1, one host sync) gives the same |M|
    as bm_set_matching + bm_match, leaves a valid maximum matching, rejects an
    invalid start without breaking the context, and restarts cleanly."""
    g = synth.rmat_graph(16, 1 << 20, seed=4)
    want = oracle_max(g)
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    cp, ri = to_dev(g)
    d_rm0, d_cm0 = torch.from_numpy(rm0).cuda(), torch.from_numpy(cm0).cuda()
    rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
    cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri) as m:
        m.set_matching(d_rm0, d_cm0)
        a = m.match()
        for _ in range(2):  # twice in a row from the same start
            b = m.match_from(d_rm0, d_cm0, rm, cm)
            assert a.card == b.card == want
            assert b.stats["initial_card"] == int((cm0 >= 0).sum())
            assert_maximum(g, rm.cpu().numpy(), cm.cpu().numpy(), b.card, want)
        r_m = int(np.flatnonzero(rm0 >= 0)[0])
        c_m = int(np.flatnonzero(cm0 >= 0)[0])
        c_free = int(np.flatnonzero(cm0 < 0)[0])
        bad_starts = []
        b = rm0.copy(); b[r_m] = -1; bad_starts.append((b, cm0))            # a row forgets its column
        b = cm0.copy(); b[c_free] = g.n_rows + 5; bad_starts.append((rm0, b))  # a column out of range
        b = rm0.copy(); b[r_m] = -3; bad_starts.append((b, cm0))            # a negative code
        b = cm0.copy(); b[c_free] = int(cm0[c_m]); bad_starts.append((rm0, b))  # two columns, one row
        for brm, bcm in bad_starts:
            with pytest.raises(bmatch.BMError) as e:
                m.match_from(torch.from_numpy(brm).cuda(), torch.from_numpy(bcm).cuda())
            assert e.value.status == bmatch.BM_ERR_INVALID_MATCHING
            assert m.match_from(d_rm0, d_cm0).card == want  # the context is still usable
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, driver=1) as h:  # the host loop's install path
        assert h.match_from(d_rm0, d_cm0).card == want
        with pytest.raises(bmatch.BMError) as e:
            h.match_from(torch.from_numpy(bad_starts[0][0]).cuda(), d_cm0)
        assert e.value.status == bmatch.BM_ERR_INVALID_MATCHING


def test_phase_limit_gives_valid_partial_matchings(c1):
    cards = []
    for k in (1, 2, 3):
        cp, ri = to_dev(c1)
        with bmatch.Matcher(c1.n_rows, c1.n_cols, c1.nnz, cp, ri, max_phases=k) as m:
            rm = torch.empty(c1.n_rows, dtype=torch.int32, device="cuda")
            cm = torch.empty(c1.n_cols, dtype=torch.int32, device="cuda")
            res = m.match(rm, cm, allow_incomplete=True)
            assert res.status == bmatch.BM_INCOMPLETE
            st, card = oracle.validate(c1.n_rows, c1.n_cols, c1.col_ptr, c1.row_idx,
                                       rm.cpu().numpy(), cm.cpu().numpy())
            assert st == 0 and card == res.card
            cards.append(card)
    assert 0 < cards[0] < cards[1] < cards[2]  # every phase with a path augments


def test_invalid_inputs_are_rejected():
    g = synth.uniform_graph(100, 100, 4, seed=1)
    cp, ri = to_dev(g)
    bad_ri = ri.clone()
    bad_ri[7] = 100  # row id out of range
    with pytest.raises(bmatch.BMError) as e:
        bmatch.Matcher(100, 100, g.nnz, cp, bad_ri)
    assert e.value.status == bmatch.BM_ERR_INVALID_CSR
    bad_cp = cp.clone()
    bad_cp[50] = bad_cp[52] + 1  # not monotone
    with pytest.raises(bmatch.BMError) as e:
        bmatch.Matcher(100, 100, g.nnz, bad_cp, ri)
    assert e.value.status == bmatch.BM_ERR_INVALID_CSR
    with bmatch.Matcher(100, 100, g.nnz, cp, ri) as m:
        rm = torch.full((100,), -1, dtype=torch.int32, device="cuda")
        cm = torch.full((100,), -1, dtype=torch.int32, device="cuda")
        rm[3] = 5  # cmatch[5] does not point back
        with pytest.raises(bmatch.BMError) as e:
            m.set_matching(rm, cm)
        assert e.value.status == bmatch.BM_ERR_INVALID_MATCHING
        res = m.match()  # the context stays usable
        assert res.card == oracle_max(g)


def test_barrier_timeout_is_reported_not_hung(c1):
    """A barrier wait limit of 1 ns runs out on the first barrier: the kernel
    records BM_ERR_TIMEOUT and every block returns; the context is then sticky
    and a fresh context works."""
    cp, ri = to_dev(c1)
    m = bmatch.Matcher(c1.n_rows, c1.n_cols, c1.nnz, cp, ri, wait_timeout_ns=1)
    with pytest.raises(bmatch.BMError) as e:
        m.match()
    assert e.value.status == bmatch.BM_ERR_TIMEOUT
    with pytest.raises(bmatch.BMError) as e:
        m.match()
    assert e.value.status == bmatch.BM_ERR_STATE
    m.close()
    rm, cm, card, _ = gpu_match(c1)
    assert card == golden_workloads()["uniform10k"]["max"]


def test_match_host_buffers(c1):
    want = golden_workloads()["uniform10k"]["max"]
    with bmatch.Matcher(c1.n_rows, c1.n_cols, c1.nnz, None, None) as m:
        rm = np.full(c1.n_rows, -1, np.int32)
        cm = np.full(c1.n_cols, -1, np.int32)
        res = m.match_host(c1.col_ptr, c1.row_idx, rm, cm)
        assert_maximum(c1, rm, cm, res.card, want)
        # second call on the same context, from a greedy start, pinned buffers
        rm0, cm0, _ = oracle.greedy(c1.n_rows, c1.n_cols, c1.col_ptr, c1.row_idx)
        prm = torch.from_numpy(rm0).pin_memory()
        pcm = torch.from_numpy(cm0).pin_memory()
        res = m.match_host(torch.from_numpy(c1.col_ptr).pin_memory(),
                           torch.from_numpy(c1.row_idx).pin_memory(), prm, pcm)
        assert_maximum(c1, prm.numpy(), pcm.numpy(), res.card, want)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["rmat21", "stencil2000"])
def test_full_size_workloads(name):
    """The benchmark's single-graph workloads at full size, GPU greedy start as
    in bench.py: |M| equals the stored Hopcroft-Karp value and the matching
    carries a Koenig certificate."""
    want = golden_workloads()[name]["max"]
    g = synth.workload(name)
    cp, ri = to_dev(g)
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri) as m:
        m.greedy()
        rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
        res = m.match(rm, cm)
    assert_maximum(g, rm.cpu().numpy(), cm.cpu().numpy(), res.card, want)


@pytest.mark.parametrize("driver", [0, 1])
def test_phase_profile_matches_counters(c1, driver):
    """The per-phase profile (Fig. 2's levels per outer iteration) adds up to
    the launch counters, and every endpoint level lies inside its phase."""
    cp, ri = to_dev(c1)
    with bmatch.Matcher(c1.n_rows, c1.n_cols, c1.nnz, cp, ri, driver=driver) as m:
        res = m.match()
        levels, ends, first, last = m.phase_profile()
    st = res.stats
    assert len(levels) == st["phases"]  # every outer iteration searched; the last found nothing
    assert int(levels.sum()) == st["levels"] and int(levels.max()) == st["max_levels_in_phase"]
    assert int(ends.sum()) == st["endpoints"]
    assert np.all((ends > 0) == (first > 0))
    assert np.all(first <= last) and np.all(last <= levels)
    assert ends[-1] == 0  # the last searching phase found no path
    assert st["final_card"] == golden_workloads()["uniform10k"]["max"]

