"""Pins for the oracle (CPU only).

Each check ties the oracle to something other than itself: exhaustive search
from the definition of a matching (Section 2 of arXiv 1303.1379), closed forms,
the Koenig/Berge characterisation of maximality, a library routine (scipy) and
the worked race example of Fig. 1.  Each is chosen so that a plausible slip in
bm_oracle.c (a dropped layer check, a wrong index, a transposed operand) fails.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_from_edges(n_rows, n_cols, edges):
    cols = [[] for _ in range(n_cols)]
    for r, c in edges:
        cols[c].append(r)
    col_ptr = np.zeros(n_cols + 1, np.int32)
    row_idx = []
    for c in range(n_cols):
        rs = sorted(set(cols[c]))
        row_idx += rs
        col_ptr[c + 1] = col_ptr[c] + len(rs)
    return col_ptr, np.array(row_idx, np.int32)


def check_maximum(n_rows, n_cols, cp, ri, rm, cm, expect):
    st, card = oracle.validate(n_rows, n_cols, cp, ri, rm, cm)
    assert st == 0 and card == expect
    st, cover = oracle.konig(n_rows, n_cols, cp, ri, rm, cm)
    assert st == 0 and cover == expect


# ------------------------------------------------------------ generators
def test_philox_known_answers():
    # Known-answer vectors of Philox-4x32-10 published with Random123.
    assert [hex(x) for x in synth.philox4x32_10([0, 0, 0, 0], [0, 0])] == \
        ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]
    assert [hex(x) for x in synth.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)] == \
        ["0x408f276d", "0x41c83b0e", "0xa20bc7c6", "0x6d5451fd"]
    assert [hex(x) for x in synth.philox4x32_10(
        [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0])] == \
        ["0xd16cfe09", "0x94fdcceb", "0x5001e420", "0x24126ea1"]


def test_generators_are_valid_csr_and_deterministic():
    g1 = synth.uniform_graph(500, 400, 8, seed=5)
    g2 = synth.uniform_graph(500, 400, 8, seed=5)
    assert np.array_equal(g1.row_idx, g2.row_idx) and np.array_equal(g1.col_ptr, g2.col_ptr)
    for g in (g1, synth.rmat_graph(10, 20000, seed=1), synth.stencil_graph(30, 90, 0.05, seed=2),
              synth.rmat_graph(10, 5000, seed=3, n=700)):
        assert oracle.csr_check(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) == 0
        for c in range(g.n_cols):  # rows sorted and distinct inside a column
            seg = g.row_idx[g.col_ptr[c]:g.col_ptr[c + 1]]
            assert np.all(np.diff(seg) > 0)
    deg = np.diff(g1.col_ptr)
    assert deg.min() >= 1 and deg.max() <= 8


def test_stencil_structure():
    g = synth.stencil_graph(40, 160, 0.05, seed=2)
    n = 1600
    # exactly 160 diagonals dropped
    diag = sum(1 for c in range(n) if c in set(g.row_idx[g.col_ptr[c]:g.col_ptr[c + 1]].tolist()))
    assert diag == n - 160
    # every entry is a 5-point neighbour
    for c in range(n):
        for r in g.row_idx[g.col_ptr[c]:g.col_ptr[c + 1]]:
            assert r - c in (0, 1, -1, 40, -40)
            if abs(r - c) == 1:
                assert r // 40 == c // 40


# ------------------------------------------------------------ brute force pins
def test_dp_equals_brute_force_all_tiny_graphs():
    # every bipartite graph on 3 rows x 3 columns, and a sample of 4 x 4
    pairs = [(r, c) for r in range(3) for c in range(3)]
    for bits in range(1 << len(pairs)):
        edges = [p for i, p in enumerate(pairs) if (bits >> i) & 1]
        cp, ri = csr_from_edges(3, 3, edges)
        assert oracle.dp_max_matching(3, cp, ri) == oracle.brute_force_max_matching(edges)
    rng = np.random.default_rng(7)
    pairs = [(r, c) for r in range(4) for c in range(4)]
    for _ in range(150):
        edges = [p for p in pairs if rng.random() < 0.35]
        cp, ri = csr_from_edges(4, 4, edges)
        assert oracle.dp_max_matching(4, cp, ri) == oracle.brute_force_max_matching(edges)


def test_hk_exhaustive_4x4_against_dp():
    # all 2^16 graphs on 4 rows x 4 columns, from empty and from greedy starts
    pairs = [(r, c) for r in range(4) for c in range(4)]
    for bits in range(1 << 16):
        edges = [p for i, p in enumerate(pairs) if (bits >> i) & 1]
        cp, ri = csr_from_edges(4, 4, edges)
        want = oracle.dp_max_matching(4, cp, ri)
        rm, cm, card, _ = oracle.hopcroft_karp(4, 4, cp, ri)
        assert card == want, edges
        if bits % 7 == 0:
            check_maximum(4, 4, cp, ri, rm, cm, want)
            g_rm, g_cm, _ = oracle.greedy(4, 4, cp, ri)
            rm, cm, card, _ = oracle.hopcroft_karp(4, 4, cp, ri, g_rm, g_cm)
            assert card == want


@pytest.mark.parametrize("seed", range(40))
def test_hk_random_rectangular_against_dp(seed):
    rng = np.random.default_rng(seed)
    nr, nc = int(rng.integers(1, 13)), int(rng.integers(1, 13))
    p = float(rng.uniform(0.05, 0.5))
    edges = [(r, c) for r in range(nr) for c in range(nc) if rng.random() < p]
    cp, ri = csr_from_edges(nr, nc, edges)
    want = oracle.dp_max_matching(nr, cp, ri)
    rm, cm, card, _ = oracle.hopcroft_karp(nr, nc, cp, ri)
    assert card == want
    check_maximum(nr, nc, cp, ri, rm, cm, want)


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("a,b", [(1, 1), (3, 7), (9, 4), (50, 50), (1, 30)])
def test_complete_bipartite(a, b):
    cp, ri = csr_from_edges(a, b, [(r, c) for r in range(a) for c in range(b)])
    rm, cm, card, _ = oracle.hopcroft_karp(a, b, cp, ri)
    assert card == min(a, b)
    check_maximum(a, b, cp, ri, rm, cm, min(a, b))


def test_permutation_matrix_and_empty():
    n = 1000
    perm = synth.permutation(n, 11, 0)
    cp, ri = csr_from_edges(n, n, [(int(perm[c]), c) for c in range(n)])
    rm, cm, card, phases = oracle.hopcroft_karp(n, n, cp, ri)
    assert card == n and phases == 1
    assert np.array_equal(cm, perm)
    cp0 = np.zeros(6, np.int32)
    rm, cm, card, _ = oracle.hopcroft_karp(4, 5, cp0, np.zeros(0, np.int32))
    assert card == 0 and np.all(rm == -1) and np.all(cm == -1)
    assert oracle.konig(4, 5, cp0, np.zeros(0, np.int32), rm, cm) == (0, 0)


def test_stencil_without_drops_is_perfect():
    g = synth.stencil_graph(60, 0, 0.0, seed=2)
    # greedy start: column j first meets row j-60 or j-1, so HK has real work
    rm, cm, c0 = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    rm, cm, card, _ = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm)
    assert card == 3600
    check_maximum(3600, 3600, g.col_ptr, g.row_idx, rm, cm, 3600)


def test_block_diagonal_batch_is_sum_of_blocks():
    b = synth.batch_graphs(24, seed=3, nr_lo=5, nr_hi=14, mu_lo=1.0, mu_hi=3.0)
    _, _, cards = oracle.hk_batch(b)
    for k in range(b.n_graphs):
        g = b.graph(k)
        assert cards[k] == oracle.dp_max_matching(g.n_rows, g.col_ptr, g.row_idx)
    # the same blocks laid out as one block-diagonal graph
    cp = [0]
    ri = []
    for k in range(b.n_graphs):
        g = b.graph(k)
        for c in range(g.n_cols):
            ri += (g.row_idx[g.col_ptr[c]:g.col_ptr[c + 1]] + int(b.row_off[k])).tolist()
            cp.append(len(ri))
    nr, nc = int(b.row_off[-1]), int(b.col_off[-1])
    _, _, card, _ = oracle.hopcroft_karp(nr, nc, np.array(cp, np.int32), np.array(ri, np.int32))
    assert card == int(cards.sum())


# ------------------------------------------------------------ CSR check
def test_csr_check_rejects_each_kind_of_bad_csr():
    """The CSR of Section 3 (cxadj / cadj): col_ptr starts at 0, never
    decreases and ends at nnz; every row id lies in [0, n_rows).  Each bad
    case below breaks exactly one of these rules and keeps the others, so
    that dropping any one test in orc_csr_check lets a case through."""
    BAD_ARG, BAD_INDEX = -1, -3
    # 3 rows, 3 columns, 4 edges: c0 {0, 2}, c1 {}, c2 {1, 2}
    cp = np.array([0, 2, 2, 4], np.int32)
    ri = np.array([0, 2, 1, 2], np.int32)
    assert oracle.csr_check(3, 3, cp, ri) == 0
    assert oracle.csr_check(3, 0, np.array([0], np.int32), np.zeros(0, np.int32)) == 0  # no columns
    assert oracle.csr_check(0, 2, np.array([0, 0, 0], np.int32), np.zeros(0, np.int32)) == 0  # no rows, no edges
    # col_ptr[0] != 0 (the rest still monotone and ending at nnz)
    assert oracle.csr_check(3, 3, np.array([1, 2, 2, 4], np.int32), ri) == BAD_ARG
    # col_ptr decreases once, starts at 0 and ends at nnz
    assert oracle.csr_check(3, 3, np.array([0, 3, 2, 4], np.int32), ri) == BAD_ARG
    assert oracle.csr_check(3, 3, np.array([0, 2, 4, 4], np.int32), ri) == 0  # same values, monotone: fine
    # col_ptr[nc] != nnz, above and below (monotone, from 0)
    assert oracle.csr_check(3, 3, np.array([0, 2, 2, 5], np.int32), ri) == BAD_ARG
    assert oracle.csr_check(3, 3, np.array([0, 2, 2, 3], np.int32), ri) == BAD_ARG
    # a row id out of range: one past the end, negative, far out
    for bad in (3, -1, 1 << 30):
        r2 = ri.copy()
        r2[3] = bad
        assert oracle.csr_check(3, 3, cp, r2) == BAD_INDEX
    r2 = ri.copy()
    r2[0] = 3  # the first edge too
    assert oracle.csr_check(3, 3, cp, r2) == BAD_INDEX
    # the bound is the row count: row 2 is out of range for 2 rows
    assert oracle.csr_check(2, 3, cp, ri) == BAD_INDEX
    # negative sizes
    assert oracle.csr_check(-1, 3, cp, ri) == BAD_ARG
    assert oracle.csr_check(3, -1, np.array([0], np.int32), ri) == BAD_ARG
    # a real generator's output stays valid; one corrupted entry anywhere is caught
    g = synth.uniform_graph(300, 250, 6, seed=12)
    assert oracle.csr_check(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) == 0
    rng = np.random.default_rng(12)
    for _ in range(20):
        r2 = g.row_idx.copy()
        r2[int(rng.integers(g.nnz))] = int(rng.choice([-2, g.n_rows, g.n_rows + 7]))
        assert oracle.csr_check(g.n_rows, g.n_cols, g.col_ptr, r2) == BAD_INDEX
        c2 = g.col_ptr.copy()
        k = int(rng.integers(1, g.n_cols))
        c2[k] = c2[k + 1] + 1  # one entry above its successor
        assert oracle.csr_check(g.n_rows, g.n_cols, c2, g.row_idx) == BAD_ARG


# ------------------------------------------------------------ certificate, validation
def test_konig_rejects_non_maximum_and_invalid():
    # path r0 - c0 - r1 - c1 : greedy takes (r0,c0), (r1,c1) => maximum 2.
    # with c0-r1 only matched, an augmenting path c1? no: build c0:{0,1}, c1:{1}
    cp, ri = csr_from_edges(2, 2, [(0, 0), (1, 0), (1, 1)])
    rm = np.array([-1, 0], np.int32)  # r1 matched to c0: c1 free, r0 free
    cm = np.array([1, -1], np.int32)
    assert oracle.validate(2, 2, cp, ri, rm, cm) == (0, 1)
    st, _ = oracle.konig(2, 2, cp, ri, rm, cm)
    assert st == -6  # augmenting path c1 - r1 - c0 - r0
    rm2, cm2, card, _ = oracle.hopcroft_karp(2, 2, cp, ri, rm, cm)
    assert card == 2 and oracle.konig(2, 2, cp, ri, rm2, cm2) == (0, 2)
    # planted errors
    assert oracle.validate(2, 2, cp, ri, np.array([1, -1], np.int32), np.array([-1, 0], np.int32))[0] == -5
    assert oracle.validate(2, 2, cp, ri, np.array([0, -1], np.int32), np.array([-1, -1], np.int32))[0] == -4
    assert oracle.validate(2, 2, cp, ri, np.array([5, -1], np.int32), np.array([-1, -1], np.int32))[0] == -3


def test_greedy_is_maximal_and_follows_column_order():
    g = synth.uniform_graph(300, 300, 4, seed=9)
    rm, cm, card = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    assert oracle.validate(300, 300, g.col_ptr, g.row_idx, rm, cm) == (0, card)
    for c in range(300):  # maximal: no edge joins two free vertices
        rows = g.row_idx[g.col_ptr[c]:g.col_ptr[c + 1]]
        if cm[c] == -1:
            assert np.all(rm[rows] != -1)
        else:  # the first row that was free when column c was visited
            first_free = [r for r in rows if rm[r] == -1 or rm[r] >= c]
            assert first_free[0] == cm[c]


def test_against_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(3):
        g = synth.uniform_graph(3000, 2600, 5, seed=seed)
        a = sp.csc_matrix((np.ones(g.nnz), g.row_idx, g.col_ptr), shape=(g.n_rows, g.n_cols))
        want = int((csgraph.maximum_bipartite_matching(a.tocsr(), perm_type="column") >= 0).sum())
        _, _, card, _ = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        assert card == want
    g = synth.rmat_graph(12, 40000, seed=1)
    a = sp.csc_matrix((np.ones(g.nnz), g.row_idx, g.col_ptr), shape=(g.n_rows, g.n_cols))
    want = int((csgraph.maximum_bipartite_matching(a.tocsr(), perm_type="column") >= 0).sum())
    rm, cm, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    _, _, card, _ = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm)
    assert card == want


# ------------------------------------------------------------ BFS levels
def load_golden(name):
    d = {"edge": [], "match": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, *v = line.split()
            v = [int(x) for x in v]
            if k in ("edge", "match"):
                d[k].append(tuple(v))
            else:
                d[k] = v if len(v) != 1 else v[0]
    return d


def test_fig1_race_example():
    d = load_golden("fig1_race.txt")
    nr, nc = d["n_rows"], d["n_cols"]
    cp, ri = csr_from_edges(nr, nc, d["edge"])
    rm = np.full(nr, -1, np.int32)
    cm = np.full(nc, -1, np.int32)
    for r, c in d["match"]:
        rm[r], cm[c] = c, r
    level, reached = oracle.bfs_levels(nr, nc, cp, ri, rm, cm, L0=2)
    assert level.tolist() == d["expect_level"]
    assert np.flatnonzero(reached).tolist() == d["expect_reached_free_rows"]
    _, _, card, _ = oracle.hopcroft_karp(nr, nc, cp, ri, rm, cm)
    assert card == d["expect_max"] == oracle.brute_force_max_matching(d["edge"])


def test_bfs_levels_against_brute_force_distances():
    # Distances by repeated relaxation over the alternating graph (Bellman-Ford
    # style, a different algorithm from the oracle's queue BFS).
    rng = np.random.default_rng(3)
    for _ in range(30):
        nr, nc = int(rng.integers(2, 30)), int(rng.integers(2, 30))
        edges = [(r, c) for r in range(nr) for c in range(nc) if rng.random() < 0.12]
        cp, ri = csr_from_edges(nr, nc, edges)
        rm, cm, _ = oracle.greedy(nr, nc, cp, ri)
        INF = 10 ** 9
        dist = [0 if cm[c] == -1 else INF for c in range(nc)]
        changed = True
        while changed:
            changed = False
            for r, c in edges:
                if dist[c] < INF and rm[r] >= 0 and dist[c] + 1 < dist[rm[r]]:
                    dist[rm[r]] = dist[c] + 1
                    changed = True
        level, reached = oracle.bfs_levels(nr, nc, cp, ri, rm, cm, L0=2)
        for c in range(nc):
            assert level[c] == (1 if dist[c] == INF else 2 + dist[c])
        want = sorted({r for r, c in edges if dist[c] < INF and rm[r] == -1})
        assert np.flatnonzero(reached).tolist() == want


def test_random_permutation_keeps_the_maximum():
    """Section 4's RCP instances: permuting rows and columns changes the
    difficulty, never the maximum matching size."""
    for g in (synth.uniform_graph(2000, 1800, 5, seed=3), synth.stencil_graph(40, 160, 0.05, seed=2),
              synth.rmat_graph(11, 15000, seed=7)):
        h = synth.permute_graph(g, seed=5)
        assert oracle.csr_check(h.n_rows, h.n_cols, h.col_ptr, h.row_idx) == 0
        assert h.nnz == g.nnz
        a = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2]
        b = oracle.hopcroft_karp(h.n_rows, h.n_cols, h.col_ptr, h.row_idx)[2]
        assert a == b
    p = synth.permutation(1000, 5, 0)
    assert sorted(p.tolist()) == list(range(1000)) and not np.array_equal(p, np.arange(1000))


def test_batch_recipe():
    """The batched workload's recipe: rows log-uniform in [100, 50,000], columns
    = rows x U[0.8, 1.25], column degrees in 1..round(2mu - 1) <= 23, every
    graph a valid CSR at its offsets, and the same batch for the same seed."""
    b = synth.batch_graphs(96, seed=3)
    b2 = synth.batch_graphs(96, seed=3)
    assert np.array_equal(b.row_idx, b2.row_idx) and np.array_equal(b.col_ptr, b2.col_ptr)
    assert b.n_rows.min() >= 100 and b.n_rows.max() <= 50_000
    ratio = b.n_cols / b.n_rows
    assert ratio.min() >= 0.8 - 1e-2 and ratio.max() <= 1.25 + 1e-2
    assert np.array_equal(np.diff(b.row_off), b.n_rows) and np.array_equal(np.diff(b.col_off), b.n_cols)
    for k in range(b.n_graphs):
        g = b.graph(k)
        assert oracle.csr_check(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) == 0
        deg = np.diff(g.col_ptr)
        assert deg.min() >= 1 and deg.max() <= 23
