/*
 * Seeded synthetic bipartite graphs in column CSR form.
 *
 * This file only draws inputs.  It holds none of the matching method's
 * arithmetic and serves the CUDA path's tests, the oracle's tests and the
 * benchmark alike.  A graph is stored the way Section 3 of Deveci, Kaya, Ucar
 * and Catalyurek (arXiv 1303.1379) stores it: cxadj/cadj, here col_ptr[nc+1]
 * and row_idx[nnz], with the rows of each column sorted and distinct.
 *
 * Every random word is a pure function of (seed, purpose, indices) computed by
 * Philox-4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Any part of a graph can therefore be regenerated
 * on its own, the output does not depend on the thread count, and a device
 * implementation of the same function yields the same graphs.
 *
 * Counter layout used throughout: ctr = (a, b, c, purpose), key = (seed low
 * 32 bits, seed high 32 bits).  "below(w, n)" maps a 32-bit word to [0, n) by
 * the multiply-shift (w * n) >> 32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BMS_EXPORT __attribute__((visibility("default")))

enum {
    P_DEG = 1,     /* column degree                           */
    P_ROW = 2,     /* candidate rows of a column              */
    P_RMAT = 3,    /* R-MAT quadrant choices                  */
    P_DIAG = 4,    /* stencil: which diagonals are dropped    */
    P_OFF = 5,     /* stencil: which off-diagonals are dropped */
    P_PARAM = 6,   /* per-graph size parameters of a batch    */
    P_PERM = 7     /* random row / column permutations        */
};

static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox-4x32 with 10 rounds, as defined by Salmon et al. (SC'11): each round
 * multiplies words 0 and 2 by two fixed odd constants, mixes the high halves
 * with the other words and the round key, and the key is bumped by two Weyl
 * constants between rounds. */
BMS_EXPORT void bms_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                                  uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static inline void draw4(uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, uint32_t c,
                         uint32_t out[4]) {
    uint32_t ctr[4] = {a, b, c, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    bms_philox4x32_10(ctr, key, out);
}

static inline uint32_t below(uint32_t w, uint32_t n) {
    return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

static void sort_i32(int32_t *v, int64_t n) {
    if (n < 32) { /* insertion sort for the common short column */
        for (int64_t i = 1; i < n; ++i) {
            int32_t x = v[i];
            int64_t j = i - 1;
            while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
            v[j + 1] = x;
        }
        return;
    }
    /* heap sort: no recursion, no allocation */
    for (int64_t start = n / 2 - 1; start >= 0; --start) {
        int64_t root = start;
        for (;;) {
            int64_t child = 2 * root + 1;
            if (child >= n) break;
            if (child + 1 < n && v[child + 1] > v[child]) ++child;
            if (v[root] >= v[child]) break;
            int32_t t = v[root]; v[root] = v[child]; v[child] = t;
            root = child;
        }
    }
    for (int64_t end = n - 1; end > 0; --end) {
        int32_t t = v[0]; v[0] = v[end]; v[end] = t;
        int64_t root = 0;
        for (;;) {
            int64_t child = 2 * root + 1;
            if (child >= end) break;
            if (child + 1 < end && v[child + 1] > v[child]) ++child;
            if (v[root] >= v[child]) break;
            int32_t u = v[root]; v[root] = v[child]; v[child] = u;
            root = child;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Uniform random bipartite graph                                       */
/*   degree of column c: 1 + below(word0 of draw(P_DEG, c, graph, 0), dmax),
 *   clamped to nr; rows: candidate k of column c is
 *   below(word k%4 of draw(P_ROW, c, graph, k/4), nr); a candidate already
 *   chosen for that column is skipped.                                 */
/* ------------------------------------------------------------------ */

static inline int32_t uniform_degree(uint64_t seed, uint32_t graph, int32_t nr, int32_t dmax,
                                     int32_t c) {
    if (nr <= 0) return 0;
    uint32_t w[4];
    draw4(seed, P_DEG, (uint32_t)c, graph, 0, w);
    int32_t d = 1 + (int32_t)below(w[0], (uint32_t)dmax);
    return d < nr ? d : nr;
}

/* Fills col_ptr[0..nc] and returns nnz (or -1 on bad arguments). */
BMS_EXPORT int64_t bms_uniform_degrees(uint64_t seed, uint32_t graph, int32_t nr, int32_t nc,
                                       int32_t dmax, int32_t *col_ptr) {
    if (nr < 0 || nc < 0 || dmax < 1 || dmax > 4096) return -1;
    int64_t acc = 0;
    col_ptr[0] = 0;
    for (int32_t c = 0; c < nc; ++c) {
        acc += uniform_degree(seed, graph, nr, dmax, c);
        if (acc > INT32_MAX) return -1;
        col_ptr[c + 1] = (int32_t)acc;
    }
    return acc;
}

static void uniform_column(uint64_t seed, uint32_t graph, int32_t nr, int32_t c, int32_t deg,
                           int32_t *out) {
    int32_t have = 0;
    uint32_t k = 0;
    uint32_t w[4];
    while (have < deg) {
        if ((k & 3u) == 0) draw4(seed, P_ROW, (uint32_t)c, graph, k >> 2, w);
        int32_t r = (int32_t)below(w[k & 3u], (uint32_t)nr);
        ++k;
        int dup = 0;
        for (int32_t i = 0; i < have; ++i)
            if (out[i] == r) { dup = 1; break; }
        if (!dup) out[have++] = r;
    }
    sort_i32(out, deg);
}

BMS_EXPORT int bms_uniform_fill(uint64_t seed, uint32_t graph, int32_t nr, int32_t nc,
                                const int32_t *col_ptr, int32_t *row_idx) {
    if (nr < 0 || nc < 0) return -1;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int32_t c = 0; c < nc; ++c)
        uniform_column(seed, graph, nr, c, col_ptr[c + 1] - col_ptr[c], row_idx + col_ptr[c]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM'04) bipartite graph         */
/*   sample i draws one 32-bit word per bit level l (from the most
 *   significant bit down): word l%4 of draw(P_RMAT, i, l/4, 0).  The word
 *   picks quadrant (row bit, column bit) = (0,0) below ta, (0,1) below tb,
 *   (1,0) below tc, else (1,1), with ta < tb < tc cumulative thresholds in
 *   units of 2^-32.  Ids >= n are rejected (dropped); duplicate edges are
 *   removed.                                                          */
/* ------------------------------------------------------------------ */

/* row_idx must have room for nsamples entries; col_ptr for n+1.  Returns nnz. */
BMS_EXPORT int64_t bms_rmat(uint64_t seed, int32_t scale, int32_t n, int64_t nsamples, double a,
                            double b, double c, int32_t *col_ptr, int32_t *row_idx) {
    if (scale < 1 || scale > 30 || n < 1 || n > (1 << scale) || nsamples < 0 ||
        nsamples > INT32_MAX)
        return -1;
    const double two32 = 4294967296.0;
    uint32_t ta = (uint32_t)floor(a * two32);
    uint32_t tb = (uint32_t)floor((a + b) * two32);
    uint32_t tc = (uint32_t)floor((a + b + c) * two32);
    int32_t *srow = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsamples ? nsamples : 1));
    int32_t *scol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsamples ? nsamples : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!srow || !scol || !cnt) { free(srow); free(scol); free(cnt); return -2; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nsamples; ++i) {
        uint32_t r = 0, cc = 0, w[4];
        for (int32_t l = 0; l < scale; ++l) {
            if ((l & 3) == 0) draw4(seed, P_RMAT, (uint32_t)i, (uint32_t)(l >> 2), 0, w);
            uint32_t u = w[l & 3];
            uint32_t rb = (u >= tb) ? 1u : 0u;          /* quadrants c, d */
            uint32_t cb = (u >= ta && u < tb) || (u >= tc) ? 1u : 0u; /* b, d */
            r = (r << 1) | rb;
            cc = (cc << 1) | cb;
        }
        if ((int64_t)r >= n || (int64_t)cc >= n) { srow[i] = -1; scol[i] = -1; }
        else { srow[i] = (int32_t)r; scol[i] = (int32_t)cc; }
    }
    /* counting sort by column (sequential: keeps sample order inside a column) */
    for (int64_t i = 0; i < nsamples; ++i)
        if (scol[i] >= 0) cnt[scol[i] + 1]++;
    for (int32_t k = 0; k < n; ++k) cnt[k + 1] += cnt[k];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n + 1);
    if (!pos) { free(srow); free(scol); free(cnt); return -2; }
    memcpy(pos, cnt, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < nsamples; ++i)
        if (scol[i] >= 0) row_idx[pos[scol[i]]++] = srow[i];
    free(pos);
    free(srow);
    free(scol);
    /* sort and deduplicate each column in place; record unique counts */
    int32_t *ucnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!ucnt) { free(cnt); return -2; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t k = 0; k < n; ++k) {
        int32_t *v = row_idx + cnt[k];
        int64_t m = cnt[k + 1] - cnt[k];
        sort_i32(v, m);
        int64_t u = 0;
        for (int64_t i = 0; i < m; ++i)
            if (u == 0 || v[i] != v[u - 1]) v[u++] = v[i];
        ucnt[k] = (int32_t)u;
    }
    /* compact (sequential, moves data left only) */
    int64_t out = 0;
    col_ptr[0] = 0;
    for (int32_t k = 0; k < n; ++k) {
        int64_t src = cnt[k];
        if (src != out) memmove(row_idx + out, row_idx + src, sizeof(int32_t) * (size_t)ucnt[k]);
        out += ucnt[k];
        col_ptr[k + 1] = (int32_t)out;
    }
    free(ucnt);
    free(cnt);
    return out;
}

/* ------------------------------------------------------------------ */
/* 5-point stencil on a g x g grid with dropped entries                 */
/*   vertex v = y*g + x; column j holds rows j-g, j-1, j, j+1, j+g (those
 *   inside the grid) in that order.  The diagonal is dropped for exactly
 *   n_diag_drop rows: the first n_diag_drop entries of a partial
 *   Fisher-Yates shuffle of 0..n-1 whose step i swaps i with
 *   i + below(word i%4 of draw(P_DIAG, i/4, 0, 0), n - i).  Off-diagonal
 *   slot s (0: -g, 1: -1, 2: +1, 3: +g) of column j is dropped when word s of
 *   draw(P_OFF, j, 0, 0) is below floor(p_off * 2^32).                   */
/* ------------------------------------------------------------------ */

/* col_ptr: n+1; row_idx: room for 5n.  Returns nnz. */
BMS_EXPORT int64_t bms_stencil(uint64_t seed, int32_t g, int32_t n_diag_drop, double p_off,
                               int32_t *col_ptr, int32_t *row_idx) {
    if (g < 1 || g > 20000) return -1;
    int64_t n = (int64_t)g * g;
    if (n_diag_drop < 0 || n_diag_drop > n || 5 * n > INT32_MAX) return -1;
    uint32_t thr = (uint32_t)floor(p_off * 4294967296.0);
    if (p_off >= 1.0) thr = 0xFFFFFFFFu;
    uint8_t *diag_keep = (uint8_t *)malloc((size_t)n);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!diag_keep || !perm) { free(diag_keep); free(perm); return -2; }
    for (int64_t i = 0; i < n; ++i) { perm[i] = (int32_t)i; diag_keep[i] = 1; }
    uint32_t w[4];
    for (int64_t i = 0; i < n_diag_drop; ++i) {
        if ((i & 3) == 0) draw4(seed, P_DIAG, (uint32_t)(i >> 2), 0, 0, w);
        int64_t j = i + below(w[i & 3], (uint32_t)(n - i));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        diag_keep[perm[i]] = 0;
    }
    free(perm);
    /* degrees */
    col_ptr[0] = 0;
    int64_t acc = 0;
    for (int64_t j = 0; j < n; ++j) {
        int32_t x = (int32_t)(j % g), y = (int32_t)(j / g);
        draw4(seed, P_OFF, (uint32_t)j, 0, 0, w);
        int32_t d = diag_keep[j];
        if (y > 0 && w[0] >= thr) d++;
        if (x > 0 && w[1] >= thr) d++;
        if (x < g - 1 && w[2] >= thr) d++;
        if (y < g - 1 && w[3] >= thr) d++;
        acc += d;
        col_ptr[j + 1] = (int32_t)acc;
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        int32_t x = (int32_t)(j % g), y = (int32_t)(j / g);
        uint32_t ww[4];
        draw4(seed, P_OFF, (uint32_t)j, 0, 0, ww);
        int32_t *o = row_idx + col_ptr[j];
        if (y > 0 && ww[0] >= thr) *o++ = (int32_t)(j - g);
        if (x > 0 && ww[1] >= thr) *o++ = (int32_t)(j - 1);
        if (diag_keep[j]) *o++ = (int32_t)j;
        if (x < g - 1 && ww[2] >= thr) *o++ = (int32_t)(j + 1);
        if (y < g - 1 && ww[3] >= thr) *o++ = (int32_t)(j + g);
    }
    free(diag_keep);
    return acc;
}

/* ------------------------------------------------------------------ */
/* Batch of uniform graphs with log-uniform sizes                       */
/*   graph k: words (w0, w1, w2) of draw(P_PARAM, k, 0, 0):
 *     nr   = floor(exp(ln lo + (ln hi - ln lo) * w0 / 2^32)), at least 1
 *     nc   = max(1, round(nr * (amin + (amax - amin) * w1 / 2^32)))
 *     mu   = mu_lo + (mu_hi - mu_lo) * w2 / 2^32
 *     dmax = max(1, round(2 mu - 1))   (column degree U{1..dmax}, mean ~ mu)
 *   and its edges are the uniform graph above with graph id k.         */
/* ------------------------------------------------------------------ */

BMS_EXPORT int bms_batch_params(uint64_t seed, int32_t n_graphs, double nr_lo, double nr_hi,
                                double aspect_lo, double aspect_hi, double mu_lo, double mu_hi,
                                int32_t *nr, int32_t *nc, int32_t *dmax) {
    if (n_graphs < 0 || nr_lo < 1 || nr_hi < nr_lo) return -1;
    const double two32 = 4294967296.0;
    const double llo = log(nr_lo), lhi = log(nr_hi);
    for (int32_t k = 0; k < n_graphs; ++k) {
        uint32_t w[4];
        draw4(seed, P_PARAM, (uint32_t)k, 0, 0, w);
        double r = floor(exp(llo + (lhi - llo) * ((double)w[0] / two32)));
        if (r < 1) r = 1;
        double asp = aspect_lo + (aspect_hi - aspect_lo) * ((double)w[1] / two32);
        double cc = floor(r * asp + 0.5);
        if (cc < 1) cc = 1;
        double mu = mu_lo + (mu_hi - mu_lo) * ((double)w[2] / two32);
        double dm = floor(2.0 * mu - 1.0 + 0.5);
        if (dm < 1) dm = 1;
        nr[k] = (int32_t)r;
        nc[k] = (int32_t)cc;
        dmax[k] = (int32_t)dm;
    }
    return 0;
}

/* Per-graph local col_ptr blocks: graph k occupies col_ptr[col_off[k] + k ..
 * col_off[k+1] + k] (nc_k + 1 entries starting at 0).  edge_count[k] gets nnz_k. */
BMS_EXPORT int bms_batch_degrees(uint64_t seed, int32_t n_graphs, const int32_t *nr,
                                 const int32_t *nc, const int32_t *dmax, const int64_t *col_off,
                                 int32_t *col_ptr, int64_t *edge_count) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
    for (int32_t k = 0; k < n_graphs; ++k) {
        int64_t e = bms_uniform_degrees(seed, (uint32_t)k, nr[k], nc[k], dmax[k],
                                        col_ptr + col_off[k] + k);
        if (e < 0) bad = 1;
        edge_count[k] = e;
    }
    return bad ? -1 : 0;
}

BMS_EXPORT int bms_batch_fill(uint64_t seed, int32_t n_graphs, const int32_t *nr,
                              const int32_t *nc, const int64_t *col_off, const int64_t *edge_off,
                              const int32_t *col_ptr, int32_t *row_idx) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t k = 0; k < n_graphs; ++k) {
        const int32_t *cp = col_ptr + col_off[k] + k;
        int32_t *ri = row_idx + edge_off[k];
        for (int32_t c = 0; c < nc[k]; ++c)
            uniform_column(seed, (uint32_t)k, nr[k], c, cp[c + 1] - cp[c], ri + cp[c]);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Random permutation of 0..n-1 (for the randomly row/column permuted
 * instances of Section 4): a full Fisher-Yates shuffle whose step i swaps
 * i with i + below(word i%4 of draw(P_PERM, i/4, which, 0), n - i).    */
/* ------------------------------------------------------------------ */

BMS_EXPORT int bms_permutation(uint64_t seed, uint32_t which, int32_t n, int32_t *perm) {
    if (n < 0) return -1;
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    uint32_t w[4];
    for (int64_t i = 0; i + 1 < n; ++i) {
        if ((i & 3) == 0) draw4(seed, P_PERM, (uint32_t)(i >> 2), which, 0, w);
        int64_t j = i + below(w[i & 3], (uint32_t)(n - i));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

BMS_EXPORT int bms_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
