/*
 * Oracle for maximum cardinality bipartite matching -- TEST INFRASTRUCTURE.
 *
 * Plain, sequential, obviously correct CPU code that the tests, the
 * benchmark's CPU baseline and the package's smoke check compare the CUDA path
 * against.  It shares no code with the CUDA path and the product never calls
 * it.  Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline load
 * this library.
 *
 * Problem (Deveci, Kaya, Ucar, Catalyurek, arXiv 1303.1379, Section 2): a
 * bipartite graph with row and column vertices, stored by columns
 * (Section 3: cxadj/cadj, here col_ptr[nc+1]/row_idx[nnz]); a matching is a
 * set of edges with no shared vertex, stored as rmatch[r] = c, cmatch[c] = r,
 * -1 for unmatched (Section 3).  The method reaches a maximum matching, whose
 * size nu(G) has a plain definition; this file computes it independently:
 *
 *   orc_greedy          the "cheap matching" initialisation of Section 4 in
 *                       its simplest form: columns in order, each takes the
 *                       first unmatched row of its adjacency list.
 *   orc_hopcroft_karp   Hopcroft-Karp (cited in Sections 1-2 as HK, the
 *                       O(sqrt(n) tau) algorithm): phases of a BFS layering
 *                       from all free columns up to the first layer that
 *                       touches a free row, then DFS in the layered graph for
 *                       a maximal set of vertex-disjoint shortest augmenting
 *                       paths, each applied as M <- M xor E(P) (Section 2).
 *   orc_validate        the definition of a matching (Section 2).
 *   orc_konig           a Koenig vertex-cover certificate of maximality: the
 *                       alternating reachability set Z from the free columns
 *                       must touch no free row (Berge, Section 2), and the
 *                       cover (C \ Z_C) u Z_R must cover every edge and have
 *                       exactly |M| vertices.
 *   orc_bfs_levels      the alternating BFS distance of every column from the
 *                       free columns for a fixed matching -- what one full
 *                       GPUBFS pass (Algorithm 2, APFB without the early break
 *                       of Algorithm 1) assigns to bfs_array, offset by L0 --
 *                       and the set of free rows that the BFS reaches.
 *   orc_hk_batch        orc_hopcroft_karp over many graphs of a batch.
 *   orc_greedy_rounds   a cheap matching in rounds of proposals (each row
 *                       takes its smallest proposer), the start that a
 *                       parallel machine reproduces exactly.
 *   orc_apfb_wr_det     the method itself -- Algorithm 1 (APFB, or APsB)
 *                       with GPUBFS-WR (Algorithm 4) keeping one endpoint per
 *                       root (the -(row) refinement of Section 3) and
 *                       Alternate (Algorithm 3) -- run one level at a time,
 *                       with each choice that the parallel version leaves to
 *                       whichever thread comes first fixed by a smallest-id
 *                       rule (the rules are listed at the function).
 *
 * All indices are int32 and the arithmetic is exact integer.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

enum {
    ORC_OK = 0,
    ORC_BAD_ARG = -1,
    ORC_NOMEM = -2,
    ORC_BAD_INDEX = -3,      /* a match entry outside [-1, n)             */
    ORC_NOT_INVERSE = -4,    /* rmatch and cmatch disagree                */
    ORC_NOT_EDGE = -5,       /* a matched pair is not an edge             */
    ORC_AUGMENTABLE = -6,    /* an augmenting path exists: not maximum     */
    ORC_UNCOVERED = -7,      /* an edge misses the Koenig cover            */
    ORC_COVER_SIZE = -8      /* cover size differs from |M|                */
};

/* CSR sanity: col_ptr starts at 0, never decreases, ends at nnz; rows in range. */
ORC_EXPORT int orc_csr_check(int32_t nr, int32_t nc, int64_t nnz, const int32_t *cp,
                             const int32_t *ri) {
    if (nr < 0 || nc < 0 || nnz < 0) return ORC_BAD_ARG;
    if (cp[0] != 0 || (int64_t)cp[nc] != nnz) return ORC_BAD_ARG;
    for (int32_t c = 0; c < nc; ++c)
        if (cp[c + 1] < cp[c]) return ORC_BAD_ARG;
    for (int64_t e = 0; e < nnz; ++e)
        if (ri[e] < 0 || ri[e] >= nr) return ORC_BAD_INDEX;
    return ORC_OK;
}

ORC_EXPORT int64_t orc_greedy(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                              int32_t *rmatch, int32_t *cmatch) {
    int64_t card = 0;
    for (int32_t r = 0; r < nr; ++r) rmatch[r] = -1;
    for (int32_t c = 0; c < nc; ++c) {
        cmatch[c] = -1;
        for (int32_t e = cp[c]; e < cp[c + 1]; ++e) {
            int32_t r = ri[e];
            if (rmatch[r] == -1) {
                rmatch[r] = c;
                cmatch[c] = r;
                ++card;
                break;
            }
        }
    }
    return card;
}

/* Is row r adjacent to column c? (linear scan: the oracle favours clarity) */
static int has_edge(const int32_t *cp, const int32_t *ri, int32_t c, int32_t r) {
    for (int32_t e = cp[c]; e < cp[c + 1]; ++e)
        if (ri[e] == r) return 1;
    return 0;
}

ORC_EXPORT int orc_validate(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                            const int32_t *rmatch, const int32_t *cmatch, int64_t *card_out) {
    int64_t rows = 0, cols = 0;
    for (int32_t r = 0; r < nr; ++r) {
        int32_t c = rmatch[r];
        if (c == -1) continue;
        if (c < 0 || c >= nc) return ORC_BAD_INDEX;
        if (cmatch[c] != r) return ORC_NOT_INVERSE;
        if (!has_edge(cp, ri, c, r)) return ORC_NOT_EDGE;
        ++rows;
    }
    for (int32_t c = 0; c < nc; ++c) {
        int32_t r = cmatch[c];
        if (r == -1) continue;
        if (r < 0 || r >= nr) return ORC_BAD_INDEX;
        if (rmatch[r] != c) return ORC_NOT_INVERSE;
        ++cols;
    }
    if (rows != cols) return ORC_NOT_INVERSE;
    if (card_out) *card_out = rows;
    return ORC_OK;
}

/* Hopcroft-Karp from the given (valid) initial matching.  Returns |M| or a
 * negative error; *phases_out gets the number of phases that augmented. */
ORC_EXPORT int64_t orc_hopcroft_karp(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                                     int32_t *rmatch, int32_t *cmatch, int64_t *phases_out) {
    const int32_t INF = INT32_MAX;
    int64_t card;
    int rc = orc_validate(nr, nc, cp, ri, rmatch, cmatch, &card);
    if (rc != ORC_OK) return rc;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
    int32_t *next_edge = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
    int32_t *stack_col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
    int32_t *stack_row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
    if (!dist || !queue || !next_edge || !stack_col || !stack_row) {
        free(dist); free(queue); free(next_edge); free(stack_col); free(stack_row);
        return ORC_NOMEM;
    }
    int64_t phases = 0;
    for (;;) {
        /* BFS layering from every free column. */
        int32_t head = 0, tail = 0;
        for (int32_t c = 0; c < nc; ++c) {
            if (cmatch[c] == -1) { dist[c] = 0; queue[tail++] = c; }
            else dist[c] = INF;
        }
        int32_t limit = INF; /* layer of the columns that touch a free row */
        while (head < tail) {
            int32_t c = queue[head++];
            if (dist[c] >= limit) continue; /* only layers below the first free row expand */
            for (int32_t e = cp[c]; e < cp[c + 1]; ++e) {
                int32_t r = ri[e];
                int32_t c2 = rmatch[r];
                if (c2 == -1) {
                    if (limit == INF) limit = dist[c];
                } else if (dist[c2] == INF) {
                    dist[c2] = dist[c] + 1;
                    queue[tail++] = c2;
                }
            }
        }
        if (limit == INF) break; /* no augmenting path: maximum (Berge) */
        ++phases;
        /* DFS from each free column inside the layered graph. */
        for (int32_t c = 0; c < nc; ++c) next_edge[c] = cp[c];
        for (int32_t root = 0; root < nc; ++root) {
            if (cmatch[root] != -1 || dist[root] != 0) continue;
            int32_t sp = 0;
            stack_col[0] = root;
            while (sp >= 0) {
                int32_t c = stack_col[sp];
                if (next_edge[c] == cp[c + 1]) { /* exhausted: dead end */
                    dist[c] = INF;
                    --sp;
                    continue;
                }
                int32_t r = ri[next_edge[c]++];
                int32_t c2 = rmatch[r];
                if (c2 == -1) {
                    if (dist[c] != limit) continue;
                    stack_row[sp] = r;
                    /* M <- M xor E(P) along the stack */
                    for (int32_t k = sp; k >= 0; --k) {
                        rmatch[stack_row[k]] = stack_col[k];
                        cmatch[stack_col[k]] = stack_row[k];
                    }
                    ++card;
                    break;
                }
                if (dist[c2] != INF && dist[c2] == dist[c] + 1 && dist[c2] <= limit) {
                    stack_row[sp] = r;
                    stack_col[++sp] = c2;
                }
            }
        }
    }
    free(dist); free(queue); free(next_edge); free(stack_col); free(stack_row);
    if (phases_out) *phases_out = phases;
    return card;
}

/* Koenig certificate.  Returns ORC_OK and *cover_out = |K| when the matching
 * is valid and maximum; an error code otherwise. */
ORC_EXPORT int orc_konig(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                         const int32_t *rmatch, const int32_t *cmatch, int64_t *cover_out) {
    int64_t card;
    int rc = orc_validate(nr, nc, cp, ri, rmatch, cmatch, &card);
    if (rc != ORC_OK) return rc;
    uint8_t *zc = (uint8_t *)calloc((size_t)nc + 1, 1);
    uint8_t *zr = (uint8_t *)calloc((size_t)nr + 1, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
    if (!zc || !zr || !queue) { free(zc); free(zr); free(queue); return ORC_NOMEM; }
    int32_t head = 0, tail = 0;
    for (int32_t c = 0; c < nc; ++c)
        if (cmatch[c] == -1) { zc[c] = 1; queue[tail++] = c; }
    rc = ORC_OK;
    while (head < tail && rc == ORC_OK) {
        int32_t c = queue[head++];
        for (int32_t e = cp[c]; e < cp[c + 1]; ++e) {
            int32_t r = ri[e];
            if (zr[r]) continue;
            zr[r] = 1;
            int32_t c2 = rmatch[r];
            if (c2 == -1) { rc = ORC_AUGMENTABLE; break; }
            if (!zc[c2]) { zc[c2] = 1; queue[tail++] = c2; }
        }
    }
    if (rc == ORC_OK) {
        int64_t size = 0;
        for (int32_t c = 0; c < nc; ++c) size += !zc[c];
        for (int32_t r = 0; r < nr; ++r) size += zr[r];
        for (int32_t c = 0; c < nc && rc == ORC_OK; ++c) {
            if (!zc[c]) continue; /* column in the cover covers its edges */
            for (int32_t e = cp[c]; e < cp[c + 1]; ++e)
                if (!zr[ri[e]]) { rc = ORC_UNCOVERED; break; }
        }
        if (rc == ORC_OK && size != card) rc = ORC_COVER_SIZE;
        if (cover_out) *cover_out = size;
    }
    free(zc); free(zr); free(queue);
    return rc;
}

/* Alternating BFS distances for a fixed matching.  level[c] = L0 + distance
 * for every column reachable from a free column (free columns have L0),
 * L0 - 1 for the others.  reached_free_row[r] = 1 for every unmatched row
 * adjacent to a reached column.  Returns the number of such rows. */
ORC_EXPORT int64_t orc_bfs_levels(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                                  const int32_t *rmatch, const int32_t *cmatch, int32_t L0,
                                  int32_t *level, uint8_t *reached_free_row) {
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
    if (!queue) return ORC_NOMEM;
    memset(reached_free_row, 0, (size_t)nr);
    int32_t head = 0, tail = 0;
    for (int32_t c = 0; c < nc; ++c) {
        if (cmatch[c] == -1) { level[c] = L0; queue[tail++] = c; }
        else level[c] = L0 - 1;
    }
    int64_t found = 0;
    while (head < tail) {
        int32_t c = queue[head++];
        for (int32_t e = cp[c]; e < cp[c + 1]; ++e) {
            int32_t r = ri[e];
            int32_t c2 = rmatch[r];
            if (c2 == -1) {
                if (!reached_free_row[r]) { reached_free_row[r] = 1; ++found; }
            } else if (level[c2] == L0 - 1) {
                level[c2] = level[c] + 1;
                queue[tail++] = c2;
            }
        }
    }
    free(queue);
    return found;
}

/* Hopcroft-Karp over a batch (graph k: local col_ptr at col_ptr + col_off[k] + k,
 * rows at row_idx + edge_off[k], matching slices at row_off[k] / col_off[k]).
 * Graphs run in parallel when OpenMP is available; each graph is sequential. */
ORC_EXPORT int orc_hk_batch(int32_t n_graphs, const int32_t *nr, const int32_t *nc,
                            const int64_t *row_off, const int64_t *col_off,
                            const int64_t *edge_off, const int32_t *col_ptr,
                            const int32_t *row_idx, int32_t *rmatch, int32_t *cmatch,
                            int32_t greedy_first, int64_t *card_out) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t k = 0; k < n_graphs; ++k) {
        const int32_t *cp = col_ptr + col_off[k] + k;
        const int32_t *ri = row_idx + edge_off[k];
        int32_t *rm = rmatch + row_off[k];
        int32_t *cm = cmatch + col_off[k];
        if (greedy_first) orc_greedy(nr[k], nc[k], cp, ri, rm, cm);
        int64_t card = orc_hopcroft_karp(nr[k], nc[k], cp, ri, rm, cm, NULL);
        if (card < 0) bad = 1;
        card_out[k] = card;
    }
    return bad ? ORC_BAD_ARG : ORC_OK;
}

/* A cheap matching that a parallel machine computes the same way every time
 * (the start of the library's deterministic option): in every round, each
 * unmatched column that still has an unmatched row proposes to the first
 * unmatched row of its list; every proposed row takes the smallest column
 * that proposed to it.  Rounds repeat until no column proposes.  The result
 * is maximal: a column stays unmatched only when all its rows are matched.
 * rmatch/cmatch in (a valid matching, usually empty) and out; returns the
 * number of rounds run (the last one without proposals not counted) or a
 * negative error code; *card_out (nullable) gets |M|. */
ORC_EXPORT int64_t orc_greedy_rounds(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                                     int32_t *rmatch, int32_t *cmatch, int64_t *card_out) {
    int32_t *pos = malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));   /* first row not yet seen matched */
    int32_t *prop = malloc(sizeof(int32_t) * (size_t)(nr ? nr : 1));  /* smallest proposer this round */
    int32_t *want = malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));  /* row proposed to this round, -1 none */
    if (!pos || !prop || !want) { free(pos); free(prop); free(want); return ORC_NOMEM; }
    for (int32_t c = 0; c < nc; ++c) pos[c] = cp[c];
    for (int32_t r = 0; r < nr; ++r) prop[r] = -1;
    int64_t rounds = 0;
    for (;;) {
        int any = 0;
        for (int32_t c = 0; c < nc; ++c) {
            want[c] = -1;
            if (cmatch[c] != -1) continue;
            while (pos[c] < cp[c + 1] && rmatch[ri[pos[c]]] != -1) ++pos[c];
            if (pos[c] == cp[c + 1]) continue;
            const int32_t r = ri[pos[c]];
            want[c] = r;
            if (prop[r] == -1 || c < prop[r]) prop[r] = c;
            any = 1;
        }
        if (!any) break;
        ++rounds;
        for (int32_t c = 0; c < nc; ++c) {
            const int32_t r = want[c];
            if (r >= 0 && prop[r] == c) { rmatch[r] = c; cmatch[c] = r; }
        }
        for (int32_t c = 0; c < nc; ++c)
            if (want[c] >= 0) prop[want[c]] = -1;
    }
    int64_t card = 0;
    for (int32_t c = 0; c < nc; ++c) card += (cmatch[c] >= 0);
    if (card_out) *card_out = card;
    free(pos); free(prop); free(want);
    return rounds;
}

/* The method of Sections 2-3 on one graph, one BFS level at a time, every
 * choice that the parallel method leaves to a race fixed by a rule:
 *   - Roots (Algorithm 1, InitBfsArray): the unmatched columns that have at
 *     least one row; each starts its own tree at level L0.
 *   - Level L (Algorithm 4 loop body): a column whose root already owns an
 *     endpoint is skipped (the GPUBFS-WR early exit); any other column scans
 *     its rows.  A matched row leads to its column; if that column is not yet
 *     in a tree it joins level L + 1, and of all level-L columns that reach it
 *     the smallest id becomes its predecessor (and gives it its root).  An
 *     unmatched row that no root owns yet offers itself to the smallest
 *     (root, column) pair that reaches it at this level.
 *   - End of level L: every root that received offers takes the smallest
 *     offering row as its one endpoint (the -(row) refinement); the other
 *     offering rows stay unmatched and may be reached again later.  A root
 *     that took an endpoint at level L stops from level L + 1 on; the columns
 *     it claimed for level L + 1 stay claimed.
 *   - The search ends after a level that claims no column (APFB), or after
 *     the first level that yields an endpoint (APsB, apsb != 0).
 *   - Alternate (Algorithm 3): every endpoint's path is walked back to its
 *     root, each column taking the row below it; the trees are disjoint, so
 *     the walks never meet.
 *   - Algorithm 1's outer loop stops after a search without endpoints, or
 *     when no root is left.
 * rmatch/cmatch: a valid initial matching in, the maximum matching out.
 * stats (nullable, 9 entries): phases (outer iterations, the final empty one
 * included), BFS levels, endpoints, columns inserted into a level, columns
 * expanded, edges scanned, scanned edges whose row was matched, Alternate
 * steps (columns rematched), roots over all searches.
 * Returns |M| or a negative error code. */
ORC_EXPORT int64_t orc_apfb_wr_det(int32_t nr, int32_t nc, const int32_t *cp, const int32_t *ri,
                                   int32_t *rmatch, int32_t *cmatch, int32_t apsb,
                                   int64_t *stats) {
    const int32_t L0 = 2;
    const size_t NC = (size_t)(nc ? nc : 1), NR = (size_t)(nr ? nr : 1);
    int32_t *clev = malloc(sizeof(int32_t) * NC);    /* level at which the column joined a tree, -1 none */
    int32_t *par = malloc(sizeof(int32_t) * NC);     /* predecessor column, -1 for a root */
    int32_t *croot = malloc(sizeof(int32_t) * NC);   /* root of the column's tree */
    int32_t *served = malloc(sizeof(int32_t) * NC);  /* per root: its endpoint row, -1 none */
    int32_t *pick = malloc(sizeof(int32_t) * NC);    /* per root: smallest offering row this level */
    int32_t *front = malloc(sizeof(int32_t) * NC);
    int32_t *next = malloc(sizeof(int32_t) * NC);
    int32_t *off_root = malloc(sizeof(int32_t) * NR);  /* offer of an unmatched row, -1 none */
    int32_t *off_col = malloc(sizeof(int32_t) * NR);
    int32_t *offered = malloc(sizeof(int32_t) * NR);   /* rows with an offer this level */
    uint8_t *owned = malloc(NR);                        /* row is some root's endpoint this search */
    int32_t *eps = malloc(sizeof(int32_t) * NR);
    int32_t *epar = malloc(sizeof(int32_t) * NR);      /* predecessor column of an endpoint */
    int64_t rc = 0;
    if (!clev || !par || !croot || !served || !pick || !front || !next || !off_root || !off_col ||
        !offered || !owned || !eps || !epar) {
        rc = ORC_NOMEM;
        goto done;
    }
    int64_t st[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int64_t searches = 0;
    int no_roots = 0;
    for (int32_t r = 0; r < nr; ++r) off_root[r] = -1;
    for (int32_t c = 0; c < nc; ++c) pick[c] = INT32_MAX;
    for (;;) {
        int32_t nf = 0;
        for (int32_t c = 0; c < nc; ++c) {
            clev[c] = -1;
            served[c] = -1;
            if (cmatch[c] == -1 && cp[c + 1] > cp[c]) {
                clev[c] = L0;
                par[c] = -1;
                croot[c] = c;
                front[nf++] = c;
            }
        }
        if (nf == 0) { no_roots = 1; break; }
        ++searches;
        st[8] += nf;
        memset(owned, 0, NR);
        int32_t nep = 0;
        for (int32_t L = L0;; ++L) {
            ++st[1];
            int32_t nn = 0, noff = 0;
            for (int32_t i = 0; i < nf; ++i) {
                const int32_t c = front[i];
                const int32_t rho = croot[c];
                if (served[rho] != -1) continue;
                ++st[4];
                for (int32_t e = cp[c]; e < cp[c + 1]; ++e) {
                    const int32_t r = ri[e];
                    const int32_t m = rmatch[r];
                    ++st[5];
                    if (m >= 0) {
                        ++st[6];
                        if (clev[m] == -1) {
                            clev[m] = L + 1;
                            par[m] = c;
                            next[nn++] = m;
                        } else if (clev[m] == L + 1 && c < par[m]) {
                            par[m] = c;
                        }
                    } else if (!owned[r]) {
                        if (off_root[r] == -1) {
                            off_root[r] = rho;
                            off_col[r] = c;
                            offered[noff++] = r;
                        } else if (rho < off_root[r] || (rho == off_root[r] && c < off_col[r])) {
                            off_root[r] = rho;
                            off_col[r] = c;
                        }
                    }
                }
            }
            for (int32_t i = 0; i < noff; ++i) {
                const int32_t r = offered[i];
                if (r < pick[off_root[r]]) pick[off_root[r]] = r;
            }
            int found = 0;
            for (int32_t i = 0; i < noff; ++i) {
                const int32_t r = offered[i];
                const int32_t rho = off_root[r];
                if (pick[rho] == r) {
                    owned[r] = 1;
                    served[rho] = r;
                    epar[r] = off_col[r];
                    eps[nep++] = r;
                    found = 1;
                }
            }
            for (int32_t i = 0; i < noff; ++i) {
                const int32_t r = offered[i];
                pick[off_root[r]] = INT32_MAX;
                off_root[r] = -1;
            }
            for (int32_t i = 0; i < nn; ++i) croot[next[i]] = croot[par[next[i]]];
            st[3] += nn;
            if (nn == 0) break;
            if (apsb && found) break;
            int32_t *t = front;
            front = next;
            next = t;
            nf = nn;
        }
        st[2] += nep;
        if (nep == 0) break;
        for (int32_t i = 0; i < nep; ++i) {
            int32_t r = eps[i];
            int32_t c = epar[r];
            for (;;) {
                const int32_t below = cmatch[c];
                cmatch[c] = r;
                rmatch[r] = c;
                ++st[7];
                if (par[c] < 0) break;
                r = below;
                c = par[c];
            }
        }
    }
    st[0] = searches + no_roots;
    if (stats) memcpy(stats, st, sizeof(st));
    for (int32_t c = 0; c < nc; ++c) rc += (cmatch[c] >= 0);
done:
    free(clev); free(par); free(croot); free(served); free(pick); free(front); free(next);
    free(off_root); free(off_col); free(offered); free(owned); free(eps); free(epar);
    return rc;
}

ORC_EXPORT int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
