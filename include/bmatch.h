/*
 * bmatch -- maximum cardinality matching in sparse bipartite graphs on one
 * GB300 GPU (sm_103a), after Deveci, Kaya, Ucar and Catalyurek, "GPU accelerated
 * maximum cardinality matching algorithms for bipartite graphs"
 * (arXiv 1303.1379).
 *
 * The method (Section 3, Algorithm 1): starting from any matching, repeat
 * phases until a phase finds no augmenting path.  A phase is a level-synchronous
 * breadth-first search that starts from every unmatched column at once
 * (GPUBFS, Algorithm 2, or GPUBFS-WR, Algorithm 4, which tracks the root of
 * every search tree and stops a tree once a path for its root is found),
 * then Alternate (Algorithm 3) flips the edges along the predecessor chains of
 * the unmatched rows that the search reached, then FixMatching (Section 3)
 * unmatches every row r with cmatch[rmatch[r]] != r.  APFB runs each search
 * until no column is added; APsB stops it at the first level that reaches an
 * unmatched row (Algorithm 1, the break inside the level loop).
 *
 * Conventions (Section 3): the graph is given by columns, CSR style:
 * the rows adjacent to column c are row_idx[col_ptr[c] .. col_ptr[c+1]-1]
 * (col_ptr has n_cols+1 entries, col_ptr[0] = 0, col_ptr[n_cols] = nnz, rows in
 * [0, n_rows); rows inside a column need not be sorted; duplicates are
 * tolerated).  A matching is rmatch[n_rows], cmatch[n_cols] with
 * rmatch[r] = c and cmatch[c] = r for a matched pair and -1 for an unmatched
 * vertex.  All indices are int32; nnz < 2^31.
 *
 * Execution: every call is issued on the stream given to bm_create and is
 * synchronous with respect to the host unless stated otherwise (it returns
 * after the work it enqueued has finished, so its status is final).  Device
 * pointers are CUDA device (or managed) addresses on the current device.
 *
 * Errors: every entry point returns BM_OK (0), BM_INCOMPLETE (1, a caller-set
 * phase limit was reached; the matching is valid but maybe not maximum) or a
 * negative BM_ERR_* code.  The library never aborts, traps or hangs the GPU:
 * every device-side wait is bounded by a time limit after which the kernel
 * returns BM_ERR_TIMEOUT.  After an error the context's outputs are undefined
 * and the error is sticky: later calls on that context return BM_ERR_STATE
 * (destroy is always allowed).
 */
#ifndef BMATCH_H
#define BMATCH_H

#include <stdint.h>

#if defined(__GNUC__)
#define BM_API __attribute__((visibility("default")))
#else
#define BM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define BM_OK 0
#define BM_INCOMPLETE 1
#define BM_ERR_INVALID_ARG (-1)  /* null pointer, negative size, bad option   */
#define BM_ERR_INVALID_CSR (-2)  /* col_ptr not monotone from 0 to nnz, or a row id outside [0, n_rows) */
#define BM_ERR_NOMEM (-3)        /* device or pinned allocation failed         */
#define BM_ERR_ITER_LIMIT (-4)   /* safety cap on phases or levels reached     */
#define BM_ERR_TIMEOUT (-5)      /* a device-side barrier wait ran out of time */
#define BM_ERR_CUDA (-6)         /* a CUDA runtime call failed                 */
#define BM_ERR_STATE (-7)        /* earlier sticky error, or calls out of order */
#define BM_ERR_UNSUPPORTED (-8)  /* device cannot run the cooperative launch   */
#define BM_ERR_INVALID_MATCHING (-9) /* initial matching out of range or rmatch/cmatch not inverse */
#define BM_ERR_TOO_LARGE (-10)   /* graph too large for bm_match_noalloc's fixed scratch */
#define BM_ERR_CHECK (-11)       /* range-checked build (libbmatch_checked.so) only: an index
                                    out of range, or rmatch/cmatch not inverse between phases */

/* Algorithm 1: APFB keeps searching until no column is inserted; APsB stops
 * at the first level that reaches an unmatched row. */
#define BM_APFB 0
#define BM_APSB 1
/* Algorithm 2 (GPUBFS) or Algorithm 4 (GPUBFS-WR, root tracking + early exit). */
#define BM_GPUBFS 0
#define BM_GPUBFS_WR 1
/* Device-resident loop over phases and levels (one cooperative launch per
 * match) or the paper's host loop (one launch per level, host reads flags). */
#define BM_DRIVER_PERSISTENT 0
#define BM_DRIVER_HOST 1

typedef struct bm_options {
    int32_t mode;          /* BM_APFB (default) or BM_APSB                                  */
    int32_t bfs;           /* BM_GPUBFS_WR (default) or BM_GPUBFS                           */
    int32_t driver;        /* BM_DRIVER_PERSISTENT (default) or BM_DRIVER_HOST              */
    int32_t wr_one_endpoint; /* GPUBFS-WR only: 1 (default) = a root accepts one endpoint,
                                whose row is kept in the root's level slot as -(row), the
                                refinement Section 3 describes for APsB-GPUBFS-WR; 0 = any
                                number of endpoints per root, the root slot set to L0-2
                                (Algorithm 4 as printed)                                   */
    int32_t max_phases;    /* 0 = no limit besides the safety cap min(n_rows,n_cols)+2;
                              > 0 = stop after that many phases with BM_INCOMPLETE          */
    int32_t block_size;    /* threads per block, 0 = default (512); multiple of 32, <= 1024 */
    int32_t blocks_per_sm; /* 0 = as many as fit (capped at 2 x 1024 threads per SM)        */
    int32_t deterministic; /* 1 = every choice the parallel search leaves to whichever thread
                              comes first is fixed by a smallest-id rule, one BFS level at a
                              time (Algorithm 4 read level-synchronously): a column reached
                              from several columns of a level takes the smallest as its
                              parent and root; an unmatched row reached by several roots
                              offers itself to the smallest (root, column); a root takes the
                              smallest row offered to it as its one endpoint, the other rows
                              stay unmatched; a root served at level L stops at level L+1.
                              bm_match, bm_match_from and bm_bfs then return the same
                              matching and counters on every run and for every block size,
                              and bm_greedy runs the cheap matching in rounds: every
                              unmatched column proposes to the first unmatched row of its
                              list, every proposed row takes the smallest proposing column,
                              until no column proposes.  Batches (bm_batch_create,
                              bm_batch_set_options) follow the same rules graph by graph
                              (their cheap matching too), for every launch geometry.  Needs
                              GPUBFS-WR, wr_one_endpoint = 1 and, for a context, the
                              persistent driver (BM_ERR_INVALID_ARG otherwise); a context
                              allocates 8*n_cols + 12*n_rows bytes on its first deterministic
                              call, a batch the same over all its graphs (BM_ERR_NOMEM if
                              that fails).  0 = default                                    */
    int64_t wait_timeout_ns;  /* limit of one device-side barrier wait; 0 = 5 s             */
    int64_t total_timeout_ns; /* limit of one match launch; 0 = 120 s                       */
    int64_t reserved[6];
} bm_options;

typedef struct bm_stats {
    int32_t status;            /* same value the call returned                              */
    int32_t phases;            /* outer iterations of Algorithm 1 (incl. the last, empty one) */
    int32_t initial_card;      /* |M| of the installed matching                            */
    int32_t final_card;        /* |M| returned                                              */
    int64_t levels;            /* BFS levels over all phases (kernel calls in Fig. 2 terms) */
    int64_t max_levels_in_phase;
    int64_t columns_expanded;  /* frontier columns taken from the queues                    */
    int64_t edges_scanned;     /* adjacency entries read by the BFS                         */
    int64_t endpoints;         /* unmatched rows claimed by the BFS over all phases         */
    int64_t fix_repairs;       /* rows and columns reset by FixMatching                      */
    int64_t inserted;          /* columns the BFS added to a level                          */
    int64_t edges_to_matched;  /* scanned edges whose row was matched                       */
    int64_t alternate_steps;   /* columns rematched by Alternate                             */
    int64_t kernel_ns;         /* device time of the persistent launch (0 for the host loop) */
    int32_t grid, block;       /* blocks and threads per block of the persistent launch
                                  (0, 0 for the host loop)                                   */
    int64_t roots;             /* search roots (unmatched columns with rows) over all phases  */
} bm_stats;

typedef struct bm_ctx bm_ctx;

/* Fills *opt with the defaults listed above. */
BM_API void bm_default_options(bm_options *opt);

/* Library version as major*10000 + minor*100 + patch. */
BM_API int32_t bm_version(void);

/* Human readable name of a status code (static string, never NULL). */
BM_API const char *bm_status_string(int32_t status);

/*
 * Creates a matching context for a graph with n_rows rows, n_cols columns and
 * nnz edges (Section 3, "Data: cxadj, cadj, nc, nr").
 *   col_ptr, row_idx: device arrays (n_cols+1 and nnz int32) borrowed by the
 *     context until bm_destroy; the caller keeps ownership and must not free
 *     or modify them meanwhile.  The CSR is validated on the device
 *     (BM_ERR_INVALID_CSR).  Pass both NULL to let the context own device
 *     storage of the given sizes, to be filled by bm_upload_csr or
 *     bm_match_host.
 *   stream: cudaStream_t to issue all work on (NULL = the legacy default stream).
 *   opt: NULL for defaults.
 * The context owns its workspace (matching, levels, roots, predecessors, one
 * (column, root) queue and a second one for the next phase's roots, the
 * endpoint list: about 4*(7*n_cols + 3*n_rows) bytes),
 * allocated here.  The matching starts empty.
 */
BM_API int32_t bm_create(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *col_ptr,
                  const int32_t *row_idx, void *stream, const bm_options *opt, bm_ctx **out);

/* Copies a host CSR (n_cols+1 and nnz int32, pinned or pageable) into the
 * context's own storage and validates it.  Only for contexts created with
 * NULL col_ptr/row_idx (else BM_ERR_STATE). */
BM_API int32_t bm_upload_csr(bm_ctx *ctx, const int32_t *h_col_ptr, const int32_t *h_row_idx);

/* Replaces the options of an existing context (same meaning as in bm_create). */
BM_API int32_t bm_set_options(bm_ctx *ctx, const bm_options *opt);

/* Cheap initial matching on the GPU (the "cheap matching" initialisation of
 * Section 4): every unmatched column scans its rows in order and claims the
 * first unmatched one with an atomic compare-and-swap.  Columns are taken in
 * three passes by degree, shortest lists first (at most 32 rows: a thread
 * each; up to 2048: a warp each, longer: a block each, dealt from lists the
 * first pass builds in the context's queue).  The result is a
 * maximal matching added to the installed one; which maximal matching it is
 * depends on thread timing.  With the deterministic option the rounds of
 * proposals described there run instead (one cooperative launch; a barrier
 * wait that runs out of time returns BM_ERR_TIMEOUT), and the result depends
 * on the graph and the installed matching only.  *card_out (host, nullable)
 * gets |M|. */
BM_API int32_t bm_greedy(bm_ctx *ctx, int32_t *card_out);

/* Installs an initial matching (Section 3: "any prior matching is given in
 * rmatch and cmatch").  rmatch (n_rows) and cmatch (n_cols) are device arrays,
 * copied; both NULL installs the empty matching.  Entries must be -1 or in
 * range and the two arrays mutual inverses (else BM_ERR_INVALID_MATCHING);
 * that every matched pair is an edge is the caller's promise, not checked. */
BM_API int32_t bm_set_matching(bm_ctx *ctx, const int32_t *rmatch, const int32_t *cmatch);

/* Copies the context's current matching to device arrays (either may be NULL). */
BM_API int32_t bm_get_matching(bm_ctx *ctx, int32_t *rmatch_out, int32_t *cmatch_out);

/*
 * Algorithm 1 (APFB or APsB with GPUBFS or GPUBFS-WR, per the options) from
 * the installed matching until no augmenting path remains, then copies the
 * maximum matching to rmatch_out (n_rows) / cmatch_out (n_cols) (device,
 * either may be NULL) and |M| to *card_out (host, nullable); *stats (host,
 * nullable) gets counters.  The context keeps the result as its installed
 * matching.
 */
BM_API int32_t bm_match(bm_ctx *ctx, int32_t *rmatch_out, int32_t *cmatch_out, int32_t *card_out,
                 bm_stats *stats);

/*
 * bm_set_matching + bm_match in one call: installs the initial matching
 * rmatch0 (n_rows) / cmatch0 (n_cols) (device arrays, copied; checked as by
 * bm_set_matching; Section 3: the method starts from any matching held in
 * rmatch / cmatch) and runs Algorithm 1 from it, with one host
 * synchronisation at the end instead of two (the match launch returns at
 * once when the check failed).  Restarting from a saved matching -- resuming,
 * or timing repeated runs -- takes this call.  Outputs as for bm_match.  An
 * invalid initial matching returns BM_ERR_INVALID_MATCHING and leaves the
 * empty matching installed; the context stays usable.
 */
BM_API int32_t bm_match_from(bm_ctx *ctx, const int32_t *rmatch0, const int32_t *cmatch0,
                             int32_t *rmatch_out, int32_t *cmatch_out, int32_t *card_out,
                             bm_stats *stats);

/*
 * One-shot call with HOST buffers: copies the CSR (h_col_ptr, h_row_idx) and
 * the initial matching (h_rmatch, h_cmatch; both NULL = empty) to the device,
 * runs bm_match, and writes the maximum matching back into h_rmatch/h_cmatch
 * (if given) and |M| into *card_out.  The context must own its CSR storage
 * (created with NULL col_ptr/row_idx).  Pinned host buffers make the copies
 * asynchronous DMA; pageable ones work too.
 */
BM_API int32_t bm_match_host(bm_ctx *ctx, const int32_t *h_col_ptr, const int32_t *h_row_idx,
                      int32_t *h_rmatch, int32_t *h_cmatch, int32_t *card_out,
                      bm_stats *stats);

/*
 * One breadth-first search of Algorithm 1 (InitBfsArray, then the level loop
 * with the context's BFS kind and mode) from the installed matching, without
 * Alternate: for inspection and testing.  Outputs (device, each nullable):
 *   level_out[n_cols]  bfs_array: L0 = 2 for unmatched columns, L0 + k for a
 *                      column inserted at level k, L0 - 1 = 1 if never reached;
 *                      under GPUBFS-WR a root whose path was found holds
 *                      -(row) (one endpoint per root) or L0 - 2 = 0.
 *   root_out[n_cols]   root column of each reached column (GPUBFS-WR), else -1.
 *   pred_out[n_rows]   column from which each reached row was entered, or -1.
 *   endpoints_out[..]  the unmatched rows the search claimed (capacity n_rows),
 *   *n_endpoints_out   (host) their number.
 * The installed matching is left unchanged.
 */
BM_API int32_t bm_bfs(bm_ctx *ctx, int32_t *level_out, int32_t *root_out, int32_t *pred_out,
               int32_t *endpoints_out, int32_t *n_endpoints_out);

/*
 * Per-phase profile of the last bm_match on this context (the quantities of
 * Fig. 2 of the paper: BFS levels -- kernel calls in the paper's host loop --
 * of every outer iteration of Algorithm 1).  For each of the first
 * min(cap, phases, 4096) phases that searched: levels[i], endpoints[i] (rows
 * claimed), first_ep_level[i] / last_ep_level[i] (1-based level at which the
 * first / last endpoint was claimed, 0 if none).  Host arrays, each nullable;
 * *n_out gets the number of entries written.
 */
BM_API int32_t bm_phase_profile(bm_ctx *ctx, int32_t cap, int32_t *levels, int32_t *endpoints,
                                int32_t *first_ep_level, int32_t *last_ep_level, int32_t *n_out);

/* Releases the context and its workspace (never the caller's buffers). */
BM_API int32_t bm_destroy(bm_ctx *ctx);

/* ------------------------------------------------------------------ batches
 * Many independent graphs matched by ONE persistent launch (the paper's
 * method per graph; the batching is this library's addition, for solvers that
 * match many matrices or diagonal blocks).  Each block of the launch runs the
 * whole method on one graph at a time, taking graphs largest first from an
 * atomic counter; graphs never wait for each other.  The launch is recorded in
 * a CUDA graph once and replayed by every bm_batch_match.
 */
typedef struct bm_batch_desc {
    int32_t n_graphs;
    int32_t reserved0;
    const int32_t *n_rows;    /* device [n_graphs]                                        */
    const int32_t *n_cols;    /* device [n_graphs]                                        */
    const int64_t *row_off;   /* device [n_graphs+1], from 0: graph k's rows are entries
                                 row_off[k] .. row_off[k+1]-1 of the batch rmatch         */
    const int64_t *col_off;   /* device [n_graphs+1], from 0: its columns in cmatch       */
    const int64_t *edge_off;  /* device [n_graphs+1], from 0: its edges in row_idx        */
    const int32_t *col_ptr;   /* device: graph k's own col_ptr (n_cols[k]+1 entries, from
                                 0) starts at col_ptr + col_off[k] + k                    */
    const int32_t *row_idx;   /* device: graph k's rows, local ids in [0, n_rows[k])      */
} bm_batch_desc;

typedef struct bm_batch_stats {
    int32_t status;            /* first non-zero per-graph status, else 0                  */
    int32_t grid, block;       /* launch geometry used                                     */
    int32_t reserved0;
    int64_t phases, levels, columns_expanded, edges_scanned, endpoints, fix_repairs,
            alternate_steps;   /* sums over the graphs                                     */
    int64_t edges_to_matched;  /* scanned edges whose row was matched (sum over graphs)    */
    int64_t inserted;          /* columns the BFS added to a level (sum over graphs)       */
    int64_t reserved[2];
} bm_batch_stats;

typedef struct bm_batch bm_batch;

/* Creates a batch over the graphs described by *desc (device arrays borrowed
 * until bm_batch_destroy).  Reads the three offset arrays back once (to size
 * the workspace and order the graphs by edge count), validates every graph's
 * CSR on the device (BM_ERR_INVALID_CSR) and allocates the workspace (about
 * 12 bytes per column and 8 per row of the whole batch).  opt: mode, bfs,
 * wr_one_endpoint, block_size, blocks_per_sm are used; NULL = defaults. */
BM_API int32_t bm_batch_create(const bm_batch_desc *desc, void *stream, const bm_options *opt,
                               bm_batch **out);

/* Changes mode / BFS kind / launch geometry (the next match re-records the launch). */
BM_API int32_t bm_batch_set_options(bm_batch *b, const bm_options *opt);

/* Matches every graph.  rmatch / cmatch: device arrays over the whole batch
 * (row_off / col_off slices, local ids), the initial matchings on entry (-1
 * for none) and the maximum matchings on return.  greedy != 0 first runs the
 * cheap matching of Section 4 inside the launch.  card_out: device
 * [n_graphs] (nullable) gets each |M|.  Returns the first per-graph error (see
 * bm_batch_graph_status) or BM_OK. */
BM_API int32_t bm_batch_match(bm_batch *b, int32_t greedy, int32_t *rmatch, int32_t *cmatch,
                              int32_t *card_out, bm_batch_stats *stats);

/* Per-graph status and phase count of the last bm_batch_match (device arrays
 * [n_graphs], each nullable). */
BM_API int32_t bm_batch_graph_status(bm_batch *b, int32_t *status_out, int32_t *phases_out);

/* Autotuner: times bm_batch_match (from the initial matching rmatch0 /
 * cmatch0, copied into rmatch_work / cmatch_work before every run, all device
 * arrays over the batch) for each candidate (block_sizes[i], blocks_per_sm[i])
 * and keeps the fastest as the batch's launch geometry.  ms_out[i] (host,
 * nullable) gets the best of `reps` runs of candidate i (negative if it cannot
 * launch); *best_out (host) the chosen index. */
BM_API int32_t bm_batch_autotune(bm_batch *b, int32_t greedy, const int32_t *rmatch0,
                                 const int32_t *cmatch0, int32_t *rmatch_work,
                                 int32_t *cmatch_work, int32_t n_candidates,
                                 const int32_t *block_sizes, const int32_t *blocks_per_sm,
                                 int32_t reps, float *ms_out, int32_t *best_out);

/* Releases the batch's workspace (never the caller's buffers). */
BM_API int32_t bm_batch_destroy(bm_batch *b);

/* ------------------------------------------------------------------ serving
 * Continuous-batching server (this library's addition around the paper's
 * method).  Requests are host CSR graphs submitted at any time.  A scheduler
 * thread admits them in arrival order when their device memory -- CSR,
 * matching and workspace, about 4*(nnz + 6*n_cols + 3*n_rows) bytes -- fits in
 * a fixed device pool and a ring slot is free, uploads them on a copy stream
 * and publishes them to persistent worker blocks on the GPU, each of which
 * matches one request at a time (cheap matching + Algorithm 1, the batched
 * path's block routine) and reports |M| back through host-mapped memory.
 * Requests that arrive while others run are taken by whichever worker frees
 * first.  Workers leave together once no worker has been busy for
 * idle_timeout_ns and are relaunched when work arrives; every device-side wait
 * is bounded.
 */
typedef struct bm_server_options {
    int64_t pool_bytes;      /* device pool for resident requests; 0 = free memory - reserve     */
    int64_t reserve_bytes;   /* left free when pool_bytes = 0 (default 2 GiB)                    */
    int32_t ring_slots;      /* requests admitted at once (default 1024)                         */
    int32_t block_size;      /* threads per worker block (default 512)                           */
    int32_t blocks_per_sm;   /* worker blocks per SM (default 2, capped by occupancy; 1 with
                                exclusive_alongside)                                          */
    int32_t mode;            /* BM_APFB (default) / BM_APSB                                      */
    int32_t bfs;             /* BM_GPUBFS_WR (default) / BM_GPUBFS                               */
    int32_t keep_results;    /* 1: keep each request's matching until bm_server_release          */
    int64_t idle_timeout_ns; /* workers leave when no block has been busy this long (default 50 ms) */
    int32_t poll_interval_us;/* scheduler sleep when idle (default 5)                             */
    int32_t exclusive_alongside; /* 1 (default): requests of at least exclusive_min_edges run on
                                    their own stream beside the workers (one block per SM each,
                                    so both stay resident and small requests do not wait behind
                                    large ones); 0: the workers leave first and the request has
                                    the whole GPU.  Sharing assumes no other kernel holds the
                                    SMs' second block slot meanwhile (another server on the same
                                    GPU, say); if one does, the large request's grid waits for
                                    it, and a wait past wait limits fails the request with
                                    BM_ERR_TIMEOUT                                             */
    int64_t exclusive_min_edges; /* requests with at least this many edges run on the single-graph
                                    persistent kernel (one after another; beside the workers or
                                    alone, see exclusive_alongside) instead of on one worker
                                    block; 0 = never (default 524,288)                        */
    int32_t deterministic;   /* 1: every request runs with bm_options.deterministic's rules, its
                                cheap matching in rounds of proposals (each row takes the smallest
                                proposing column), on a worker block or on the single-graph
                                kernel alike: a request's matching depends on its graph only,
                                alone or in any mix.  Each request takes 8*n_cols + 12*n_rows
                                more bytes of the pool.  Needs bfs = BM_GPUBFS_WR.
                                0 = default                                                 */
    int32_t reserved0;
    int64_t reserved[2];
} bm_server_options;

/* Request states reported by bm_server_poll / bm_server_wait. */
#define BM_REQ_PENDING 0
#define BM_REQ_UPLOADING 1
#define BM_REQ_RUNNING 2
#define BM_REQ_DONE 3
#define BM_REQ_CANCELLED 4

typedef struct bm_request_info {
    int32_t state;       /* BM_REQ_*                                                    */
    int32_t status;      /* when done: BM_OK, BM_ERR_INVALID_CSR, BM_ERR_TOO_LARGE, ... */
    int32_t card;        /* when done: |M|                                              */
    int32_t phases;
    int64_t latency_ns;  /* when done: submit -> completion seen by the scheduler     */
    int64_t reserved[2];
} bm_request_info;

typedef struct bm_server_stats {
    int64_t pending, inflight, completed, rejected, worker_launches, pool_bytes, pool_used;
    int32_t grid, block;
    int64_t exclusive_runs;  /* requests that ran alone on the whole GPU */
    int64_t reserved[1];
} bm_server_stats;

typedef struct bm_server bm_server;

BM_API void bm_server_default_options(bm_server_options *opt);
/* Allocates the pool and the host-mapped ring, starts the scheduler thread. */
BM_API int32_t bm_server_create(const bm_server_options *opt, bm_server **out);
/* Queues a request (host CSR, pinned preferred; the buffers must stay valid
 * and unchanged until the request is done or cancelled).  *id_out gets its id.
 * A request too large for the pool is completed at once with BM_ERR_TOO_LARGE;
 * a malformed CSR completes with BM_ERR_INVALID_CSR (checked on the GPU). */
BM_API int32_t bm_server_submit(bm_server *s, int32_t n_rows, int32_t n_cols, int64_t nnz,
                                const int32_t *h_col_ptr, const int32_t *h_row_idx,
                                int32_t greedy, int64_t *id_out);
/* Non-blocking state of a request. */
BM_API int32_t bm_server_poll(bm_server *s, int64_t id, bm_request_info *info);
/* Waits up to timeout_ns for a request to finish (BM_ERR_TIMEOUT otherwise). */
BM_API int32_t bm_server_wait(bm_server *s, int64_t id, int64_t timeout_ns, bm_request_info *info);
/* Cancels a request that has not been admitted yet (else BM_ERR_STATE). */
BM_API int32_t bm_server_cancel(bm_server *s, int64_t id);
/* Copies a finished request's matching to host arrays (needs keep_results). */
BM_API int32_t bm_server_fetch(bm_server *s, int64_t id, int32_t *h_rmatch, int32_t *h_cmatch);
/* Forgets a finished or cancelled request and frees its pool memory. */
BM_API int32_t bm_server_release(bm_server *s, int64_t id);
BM_API int32_t bm_server_get_stats(bm_server *s, bm_server_stats *st);
/* Stops the scheduler and the workers and frees everything. */
BM_API int32_t bm_server_destroy(bm_server *s);

/*
 * Allocation-free matching (no counterpart in the paper; an addition for
 * callers that may not allocate).
 *
 * Some callers cannot call cudaMalloc: code running inside a memory pool or
 * arena that owns all device memory of the process, plugins whose host
 * application forbids allocation after start-up, and real-time loops where an
 * allocation could block or fail mid-run.  This entry point runs the same
 * persistent matching kernel as bm_match (APFB, GPUBFS-WR, one endpoint per
 * root) with no context and no allocation: its working arrays live in one
 * file-scope device array of BM_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads this library holds until the process exits.
 *
 *   col_ptr, row_idx  device CSR of the columns, as for bm_create (read only).
 *   rmatch, cmatch    device arrays (n_rows, n_cols): the initial matching on
 *                     entry (-1 everywhere for none), the maximum matching on
 *                     return.  Caller-owned.
 *   stream            cudaStream_t for all work (NULL = legacy default stream).
 *   card_out          host, nullable: |M|.
 * Size limit: 1024 bytes of control block plus five arrays, each rounded up
 * to a multiple of 256 bytes -- 4*n_cols (levels), 4*n_cols (roots),
 * 4*n_rows (predecessors), 8*n_cols (queue), 4*n_rows (endpoints) -- must fit
 * in BM_NOALLOC_SCRATCH_BYTES (about 1024 + 4*(4*n_cols + 2*n_rows); square
 * graphs up to n = 1,398,016), else BM_ERR_TOO_LARGE is returned before any
 * GPU work.  Invalid CSR or matching: BM_ERR_INVALID_CSR /
 * BM_ERR_INVALID_MATCHING (rmatch/cmatch unchanged then).
 * The call is synchronous: it returns after the work finished, reading the
 * result through a pageable host copy and a stream synchronisation, so it
 * cannot be captured in a CUDA graph and must not be called while a stream
 * capture is active.  The first call on a device finds the scratch array's
 * device address (cudaGetSymbolAddress) and the launch size, and keeps them
 * for the life of the process: do not use this entry point across a
 * cudaDeviceReset.  The 32 MiB are reserved on each device when the library's
 * device code is loaded there, which with lazy module loading may be the first
 * call; calls allocate nothing (no cudaMalloc, cudaFree or library routine
 * that allocates).  All calls share the one scratch array, which keeps the
 * previous call's contents (the parts that must start at zero are cleared by
 * each call): calls that overlap on the GPU -- concurrent calls on different
 * streams or host threads -- race and must be serialised by the caller.
 */
#define BM_NOALLOC_SCRATCH_BYTES (32u << 20)
BM_API int32_t bm_match_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                const int32_t *col_ptr, const int32_t *row_idx,
                                int32_t *rmatch, int32_t *cmatch, void *stream,
                                int32_t *card_out);

#ifdef __cplusplus
}
#endif

#endif /* BMATCH_H */
