"""Pins for the oracle's level-by-level run of the method with fixed tie-break
rules (orc_apfb_wr_det; CPU only).

What fixes it from outside: the maximum matching size (Hopcroft-Karp, the DP
over row subsets), the Koenig certificate, closed forms on graphs whose every
step can be worked out by hand (the diagonal, the complete bipartite graph),
two small worked examples whose results depend on each tie-break rule, and
the rules' independence from the order in which a column lists its rows.
"""
import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import synth


def csr(n_cols, adj):
    """col_ptr, row_idx from per-column row lists (order kept)."""
    cp = np.zeros(n_cols + 1, np.int32)
    for c in range(n_cols):
        cp[c + 1] = cp[c] + len(adj[c])
    ri = np.array([r for c in range(n_cols) for r in adj[c]], np.int32)
    return cp, ri


def check_maximum(nr, nc, cp, ri, rm, cm, expect):
    st, card = oracle.validate(nr, nc, cp, ri, rm, cm)
    assert st == 0 and card == expect
    st, cover = oracle.konig(nr, nc, cp, ri, rm, cm)
    assert st == 0 and cover == expect


def test_diagonal_closed_form():
    # Column c has the single row c.  One search: every root offers its own
    # row at the first level, takes it and the walk is one step long.  The
    # second outer iteration finds no root left.
    n = 7
    cp, ri = csr(n, [[c] for c in range(n)])
    rm, cm, card, st = oracle.apfb_wr_det(n, n, cp, ri)
    assert card == n and list(rm) == list(range(n)) and list(cm) == list(range(n))
    assert st == dict(phases=2, levels=1, endpoints=n, inserted=0, columns_expanded=n,
                      edges_scanned=n, edges_to_matched=0, alternate_steps=n, roots=n)


@pytest.mark.parametrize("a,b", [(1, 1), (3, 7), (7, 3), (5, 5), (1, 9), (9, 1)])
def test_complete_bipartite_closed_form(a, b):
    # K_{a,b} with a rows and b columns, from the empty matching.  Search k
    # (k = 0, 1, ...): the roots are columns k.., every free row is reached
    # by every root and offers itself to the smallest, root k, which takes the
    # smallest free row, row k.  Search 0 has one level; later searches also
    # claim the matched columns 0..k-1 (for root k, the smallest parent) and
    # stop at their level, their root being served.  When columns remain
    # after the rows run out, one more search claims all matched columns,
    # expands them and finds nothing.
    n = min(a, b)
    cp, ri = csr(b, [list(range(a)) for _ in range(b)])
    rm, cm, card, st = oracle.apfb_wr_det(a, b, cp, ri)
    assert card == n
    assert list(cm[:n]) == list(range(n)) and all(x == -1 for x in cm[n:])
    assert list(rm[:n]) == list(range(n)) and all(x == -1 for x in rm[n:])
    extra = b > a
    assert st["phases"] == n + 1
    assert st["endpoints"] == n and st["alternate_steps"] == n
    assert st["levels"] == 1 + 2 * (n - 1) + (2 if extra else 0)
    assert st["inserted"] == sum(range(1, n)) + (a if extra else 0)
    check_maximum(a, b, cp, ri, rm, cm, n)


def test_smallest_parent_takes_a_shared_column():
    # Rows 0-1, columns 0-2; row 0 is matched to column 2.  Columns 0 and 1
    # are roots and both reach column 2 through row 0 at the first level;
    # column 2 reaches the free row 1.  The smaller parent, column 0, gives
    # column 2 its root, so root 0 gets the path 0 -> row 0 -> 2 -> row 1;
    # root 1 then searches alone, claims column 0, expands it (its only row
    # leads back into the tree) and stops empty.
    cp, ri = csr(3, [[0], [0], [0, 1]])
    rm0 = np.array([2, -1], np.int32)
    cm0 = np.array([-1, -1, 0], np.int32)
    rm, cm, card, st = oracle.apfb_wr_det(2, 3, cp, ri, rm0, cm0)
    assert card == 2 and list(rm) == [0, 2] and list(cm) == [0, -1, 1]
    assert st == dict(phases=2, levels=4, endpoints=1, inserted=2, columns_expanded=5,
                      edges_scanned=6, edges_to_matched=5, alternate_steps=2, roots=3)
    check_maximum(2, 3, cp, ri, rm, cm, 2)


def test_an_offer_not_taken_stays_open():
    # Rows 0-2, columns 0-2; row 2 is matched to column 2.  Root 0 reaches
    # the free rows 0 and 1 at the first level and takes the smaller, row 0;
    # row 1 stays free.  Root 1 reaches column 2 through row 2 at the first
    # level and, one level later, row 1 (an offer nobody took).
    cp, ri = csr(3, [[0, 1], [2], [2, 1]])
    rm0 = np.array([-1, -1, 2], np.int32)
    cm0 = np.array([-1, -1, 2], np.int32)
    rm, cm, card, st = oracle.apfb_wr_det(3, 3, cp, ri, rm0, cm0)
    assert card == 3 and list(rm) == [0, 2, 1] and list(cm) == [0, 2, 1]
    assert st == dict(phases=2, levels=2, endpoints=2, inserted=1, columns_expanded=3,
                      edges_scanned=5, edges_to_matched=2, alternate_steps=3, roots=2)


def test_apsb_stops_at_the_first_level_with_an_endpoint():
    # The graph of the previous test under APsB: the first level yields root
    # 0's endpoint, so the search stops there; root 1 finds its path (now
    # through column 2 and row 1) in the next search.
    cp, ri = csr(3, [[0, 1], [2], [2, 1]])
    rm0 = np.array([-1, -1, 2], np.int32)
    cm0 = np.array([-1, -1, 2], np.int32)
    rm, cm, card, st = oracle.apfb_wr_det(3, 3, cp, ri, rm0, cm0, apsb=True)
    assert card == 3 and list(rm) == [0, 2, 1] and list(cm) == [0, 2, 1]
    assert st["phases"] == 3 and st["endpoints"] == 2 and st["levels"] == 3


@pytest.mark.parametrize("seed", range(30))
def test_tiny_graphs_reach_the_dp_maximum(seed):
    rng = np.random.default_rng(100 + seed)
    nr, nc = int(rng.integers(1, 12)), int(rng.integers(1, 12))
    p = float(rng.uniform(0.05, 0.6))
    adj = [[r for r in range(nr) if rng.random() < p] for _ in range(nc)]
    cp, ri = csr(nc, adj)
    want = oracle.dp_max_matching(nr, cp, ri)
    for apsb in (False, True):
        rm, cm, card, _ = oracle.apfb_wr_det(nr, nc, cp, ri, apsb=apsb)
        assert card == want
        check_maximum(nr, nc, cp, ri, rm, cm, want)


@pytest.mark.parametrize("nr,nc,dmax,seed", [(300, 300, 4, 1), (500, 200, 6, 2), (200, 500, 3, 3),
                                             (2000, 2000, 8, 4), (1000, 1000, 2, 5)])
def test_random_graphs_reach_the_hk_maximum(nr, nc, dmax, seed):
    g = synth.uniform_graph(nr, nc, dmax, seed=seed)
    _, _, want, _ = oracle.hopcroft_karp(nr, nc, g.col_ptr, g.row_idx)
    g_rm, g_cm, _ = oracle.greedy(nr, nc, g.col_ptr, g.row_idx)
    for start in ((None, None), (g_rm, g_cm)):
        for apsb in (False, True):
            rm, cm, card, st = oracle.apfb_wr_det(nr, nc, g.col_ptr, g.row_idx, *start, apsb=apsb)
            assert card == want
            check_maximum(nr, nc, g.col_ptr, g.row_idx, rm, cm, want)
            assert st["endpoints"] == want - (0 if start[0] is None else int((g_cm >= 0).sum()))


def test_rules_do_not_depend_on_the_order_of_a_columns_rows():
    # Every choice is a minimum over a set, so listing each column's rows in
    # reverse (or shuffled) order must give the same matching and counters.
    g = synth.rmat_graph(12, 1 << 15, seed=7)
    nr, nc = g.n_rows, g.n_cols
    g_rm, g_cm, _ = oracle.greedy(nr, nc, g.col_ptr, g.row_idx)
    base = oracle.apfb_wr_det(nr, nc, g.col_ptr, g.row_idx, g_rm, g_cm)
    rng = np.random.default_rng(0)
    for how in ("reverse", "shuffle"):
        ri = g.row_idx.copy()
        for c in range(nc):
            seg = ri[g.col_ptr[c]:g.col_ptr[c + 1]]
            if how == "reverse":
                seg[:] = seg[::-1].copy()
            else:
                rng.shuffle(seg)
        # the greedy start must not change with the order: reuse the saved one
        other = oracle.apfb_wr_det(nr, nc, g.col_ptr, ri, g_rm, g_cm)
        assert np.array_equal(base[0], other[0]) and np.array_equal(base[1], other[1])
        assert base[2] == other[2] and base[3] == other[3]


# ------------------------------------------------------------ cheap matching in rounds
def test_greedy_rounds_closed_forms():
    # K_{a,b}: every round all unmatched columns propose to the first free row,
    # which takes the smallest of them -- column k gets row k in round k + 1.
    for a, b in [(1, 1), (4, 6), (6, 4), (5, 5)]:
        cp, ri = csr(b, [list(range(a)) for _ in range(b)])
        rm, cm, card, rounds = oracle.greedy_rounds(a, b, cp, ri)
        n = min(a, b)
        assert card == n and rounds == n
        assert list(cm[:n]) == list(range(n)) and all(x == -1 for x in cm[n:])
    # a permutation: first choices never collide, one round
    perm = [3, 0, 4, 1, 2]
    cp, ri = csr(5, [[perm[c], (perm[c] + 1) % 5] for c in range(5)])
    rm, cm, card, rounds = oracle.greedy_rounds(5, 5, cp, ri)
    assert rounds == 1 and card == 5 and list(cm) == perm


def test_greedy_rounds_worked_examples():
    # Columns 0 and 1 both propose to row 0 first; row 0 takes column 0.
    # Column 1's other row (1) went to column 2 in the same round, so column
    # 1 ends unmatched, where the column-order greedy would have matched all.
    cp, ri = csr(3, [[0], [0, 1], [1, 2]])
    rm, cm, card, rounds = oracle.greedy_rounds(3, 3, cp, ri)
    assert (list(rm), list(cm), card, rounds) == ([0, 2, -1], [0, -1, 1], 2, 1)
    assert oracle.greedy(3, 3, cp, ri)[2] == 3
    # The loser of round 1 moves on to its next free row in round 2.
    cp, ri = csr(2, [[0, 1], [0, 2]])
    rm, cm, card, rounds = oracle.greedy_rounds(3, 2, cp, ri)
    assert (list(rm), list(cm), card, rounds) == ([0, -1, 1], [0, 2], 2, 2)
    # A matched column does not propose; its row is not free.
    rm0 = np.array([-1, -1, 1], np.int32)
    cm0 = np.array([-1, 2], np.int32)
    rm, cm, card, rounds = oracle.greedy_rounds(3, 2, cp, ri, rm0, cm0)
    assert (list(rm), list(cm), card, rounds) == ([0, -1, 1], [0, 2], 2, 1)


@pytest.mark.parametrize("seed", range(12))
def test_greedy_rounds_is_a_maximal_matching(seed):
    rng = np.random.default_rng(200 + seed)
    nr, nc = int(rng.integers(1, 400)), int(rng.integers(1, 400))
    g = synth.uniform_graph(nr, nc, int(rng.integers(1, 9)), seed=seed)
    rm, cm, card, rounds = oracle.greedy_rounds(nr, nc, g.col_ptr, g.row_idx)
    st, c = oracle.validate(nr, nc, g.col_ptr, g.row_idx, rm, cm)
    assert st == 0 and c == card
    for col in range(nc):
        if cm[col] == -1:  # maximal: every row of an unmatched column is matched
            assert all(rm[r] >= 0 for r in g.row_idx[g.col_ptr[col]:g.col_ptr[col + 1]])
    assert rounds <= nc
