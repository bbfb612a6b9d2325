// Device-side building blocks of the matching path (sm_103a).
//
// One phase of Algorithm 1 of arXiv 1303.1379 (Section 3) is
//   InitBfsArray -> BFS levels (Algorithm 2 GPUBFS / Algorithm 4 GPUBFS-WR)
//   -> Alternate (Algorithm 3) -> FixMatching.
// This header holds those steps as device functions over "all blocks of the
// grid", so that the persistent kernel (one launch per match, grid barriers
// between steps) and the per-step kernels of the host-driven loop run the
// same code.
//
// GB300 design (differences from the paper's Fermi kernels):
//  * The paper sweeps all nc columns at every level and tests
//    bfs_array[c] == level.  Here the columns inserted at each level are
//    appended to one per-phase queue; a level expands only its own queue
//    segment, so a level costs O(frontier + its edges), not O(nc).
//  * Insertions are claimed with a test-then-CAS on the column's level entry;
//    the single winner writes pred/root and appends the column.  The paper's
//    atomic-free writes let several threads insert the same column; a queue
//    needs exactly one.  The persistent kernel of a context claims the
//    column's matched row instead (below), one dependent load earlier.
//  * A matched column is reached only through its matched row, so "column c
//    visited" is "row cmatch[c] claimed".  With a row-indexed stamp array
//    rvis (stamp = a number unique to the phase, growing across phases and
//    calls), a level of at most RV_MAX_Q columns claims with
//    atomicMax(rvis[r], stamp), issued blind together with the rmatch[r]
//    load: one dependent round trip less than load-rmatch-then-CAS-level on
//    the deep, narrow, latency-bound levels.  Larger levels, which are
//    bandwidth-bound, claim on the column's level as before (measured faster
//    there) and their winners also stamp the row, so both kinds of level see
//    the same visited set; every winner writes the column's level.
//  * Free rows are claimed with a CAS -1 -> -2 on rmatch (the paper's plain
//    store of -2), so every endpoint has exactly one predecessor and is
//    appended once to an endpoint list; Alternate walks that list instead of
//    scanning all rows for -2.
//  * Load balance: a block takes a tile of queue entries (tiles are handed out
//    by an atomic counter), computes a block-wide prefix sum of their degrees
//    and then every thread handles edges tid, tid + blockDim, ... of the
//    tile's concatenated adjacency, ILP edges at a time (independent loads in
//    flight), finding each edge's column by binary search in shared memory.
//    A column of degree 60,000 and a column of degree 1 cost the same per edge.
//  * Appends go to a per-block shared-memory buffer that is flushed with one
//    global atomic per tile.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>

namespace bmd {

namespace cg = cooperative_groups;

constexpr int L0 = 2;  // BFS start level (Section 3 chooses L0 = 2)
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_BLOCK = 1024;
constexpr int QBUF = 2048;  // per-block append buffer (entries)
constexpr int ILP = 4;      // edges per thread in flight
constexpr int HUB_DEG = 256;  // warp-level expansion: columns of more edges are expanded by the whole block
constexpr int HUB_MAX = 16;   // ... at most this many per level (the rest stay with their warp)
constexpr int RV_MAX_Q = 32768;  // largest level (columns) that claims through row stamps

// Control block in device memory, cleared before every launch.  Per-step
// counters rotate over three slots: step s appends to slot s % 3 and clears
// slot (s + 1) % 3, which nobody reads during step s (it was last read right
// after the barrier that ended step s - 2).
struct alignas(128) Ctl {
    // grid barrier: arrival words rotate over barriers b % 3; each arrival adds
    // 1 + (block has endpoints) << 11 + (block's appended columns) << 22, and
    // the barrier is complete when the low 11 bits reach gridDim.x
    unsigned long long arrive[3][16];
    int32_t qcnt[3];           // columns appended during a step (queue positions)
    int32_t ecnt[3];           // init: unmatched columns counted during a step
    int32_t icnt[3];           // init: unmatched columns without rows counted during a step
    int32_t tcnt[3];           // tiles handed out during a step
    int32_t ep_phase;          // endpoints appended in the current phase (positions)
    int32_t err;               // first error code (0 = none)
    int32_t status;            // final status of the launch
    int32_t card;              // |M| at the end
    int32_t initial_card;
    int32_t phases;            // outer iterations of Algorithm 1, the last (empty) one included
    int32_t n_endpoints_last;  // endpoints of the last BFS (inspection)
    int32_t searches;          // breadth-first searches run (entries of the phase profile)
    int32_t dcnt[3];           // deterministic option: rows listed in ecand during a step
    int32_t ep_alt;            // the persistent one-endpoint kernel's even phases count their endpoints
                               // here (odd ones in ep_phase), so that each phase's counter can be
                               // cleared during the phase before it
    int32_t pad1[6];
    long long levels;
    long long max_levels;
    long long cols_expanded;
    long long edges_scanned;
    long long endpoints;
    long long fix_repairs;
    long long inserted;        // columns added to the queues by the BFS
    long long edges_matched;   // visited edges whose row was matched
    long long alt_steps;       // Alternate steps (columns rematched)
    long long kernel_ns;       // duration of the persistent launch (%globaltimer)
    long long roots;           // search roots over all phases
};

struct Params {
    int32_t nr, nc;
    const int32_t* __restrict__ col_ptr;
    const int32_t* __restrict__ row_idx;
    int32_t* rmatch;
    int32_t* cmatch;
    int32_t* level;      // bfs_array of the paper
    int32_t* root;       // root array of GPUBFS-WR
    int32_t* pred;       // predecessor array
    int2* queue;         // (column, root) of the current phase, level by level
    int2* queue2;        // second queue buffer: roots of the next phase (nullable)
    int32_t* endpoints;  // rows claimed as path ends in the current phase
    int32_t* rvis;       // per row: stamp of the phase that claimed its column (nullable: level-based claims)
    int2* crec;          // per column inserted this phase: (parent column, matched row); roots (-1, -1) (nullable)
    Ctl* ctl;
    int32_t mode;        // 0 APFB, 1 APsB
    int32_t one_ep;      // GPUBFS-WR: one endpoint per root (-(row) in the root slot)
    int32_t max_phases;  // stop after this many phases (>= 1)
    int32_t phase_limit_is_error;
    int32_t bfs_only;    // run one BFS, no Alternate, leave the matching as installed
    int32_t profile_cap; // phases recorded in `profile`
    int32_t* profile;    // per phase: levels, endpoints, first and last level with an endpoint (nullable)
    long long wait_ns;   // limit of one barrier wait
    long long total_ns;  // limit of the whole launch
    int32_t stamp_base;  // rvis stamp of phase k is stamp_base + k (k >= 1); above every stamp in rvis
    int32_t* chk;        // range-checked build: error word set when an index is out of range (nullable)
    // deterministic option (nullable otherwise): per column the tree-entry key
    // (level << 32 | parent), per row the offer key (root << 32 | column), and
    // the rows that received an offer during the current level
    unsigned long long* dkey;
    unsigned long long* ekey;
    int32_t* ecand;
    // one block per graph, one endpoint per root (SB instantiations): bitmaps in shared
    // memory of the columns already in a tree and of the roots already served, in place of
    // the level array's tests and claims
    unsigned* vis;
    unsigned* srv;
};

// Per-block shared state of the steps.
struct Smem {
    int tile;
    int qn;     // appends since the last flush (may exceed QBUF: the excess went to global memory)
    int qbase;  // global position of the flushed buffer
    int total;  // edges of the current tile
    int npush;  // columns this block appended during the current step
    int has_ep; // this block appended an endpoint during the current step
    int bc_a, bc_b, bc_c, bc_d, ok;  // barrier broadcast
    int grab[2];  // warp-level expansion: queue positions handed out, by level parity
    int nhub[2];  // warp-level expansion: columns set aside for the whole block, by level parity
    int hub[4][HUB_MAX];  // their column, root, first edge and degree
    int wsum[32];
    int off[MAX_BLOCK];  // exclusive prefix of the tile's degrees
    int beg[MAX_BLOCK];  // first edge of each tile column
    int col[MAX_BLOCK];  // column, or -1 if its root is already served
    int root[MAX_BLOCK];
    int2 qbuf[QBUF];
};

// ------------------------------------------------------------------ memory helpers
__device__ __forceinline__ int ld_volatile(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile(int32_t* p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_error(Ctl* ctl, int code) { atomicCAS(&ctl->err, 0, code); }

// Range-checked build (compiled with BM_CHECKED, the library libbmatch_checked.so):
// every index the steps compute from data (a row id, a matched column, a root,
// a queue entry) is checked before it is used; an index out of range records
// BM_ERR_CHECK (-11) in p.chk and the access is skipped, so a fault in the
// method's bookkeeping shows as a status instead of a stray memory access.
// In the normal build the checks compile to nothing.
#ifdef BM_CHECKED
__device__ __forceinline__ bool idx_ok(const Params& p, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    if (p.chk) atomicCAS(p.chk, 0, -11 /*BM_ERR_CHECK*/);
    return false;
}
#else
__device__ __forceinline__ bool idx_ok(const Params&, long long, long long) { return true; }
#endif

// CSR reads: through the read-only (non-coherent) path when the CSR cannot
// change during the kernel (NC), else through L2 only.
template <bool NC>
__device__ __forceinline__ int ld_csr(const int32_t* p) {
    if (NC) return __ldg(p);
    return __ldcg(p);
}

// Shared-memory bitmaps of the one-block-per-graph routine (p.vis, p.srv).
constexpr int SB_MAX_COLS = 61440;  // columns a graph may have for the bitmaps (7.5 KB each; with the
                                    // shared state the block stays within 48 KB of static shared memory)
__device__ __forceinline__ bool sb_test(const unsigned* b, int i) {
    return (((const volatile unsigned*)b)[i >> 5] >> (i & 31)) & 1u;
}
// Sets bit i; true if this call set it (it was clear).
__device__ __forceinline__ bool sb_claim(unsigned* b, int i) {
    const unsigned m = 1u << (i & 31);
    return !(atomicOr(&b[i >> 5], m) & m);
}

// Appends v at base + (running count of `slot`) with one atomic per group of
// converged lanes (endpoints, and columns when the block buffer is full).
template <class T>
__device__ __forceinline__ void push(T* buf, int base, int32_t* slot, T v) {
    cg::coalesced_group g = cg::coalesced_threads();
    int pos = 0;
    if (g.thread_rank() == 0) pos = atomicAdd(slot, (int)g.size());
    pos = g.shfl(pos, 0) + (int)g.thread_rank();
    buf[base + pos] = v;
}

// Appends a (column, root) entry to the block's buffer (global fallback when it is full).
__device__ __forceinline__ void push_block(const Params& p, int2* q, Smem& sm, int qbase, int slot, int2 v) {
    const int pos = atomicAdd(&sm.qn, 1);
    if (pos < QBUF) sm.qbuf[pos] = v;
    else push(q, qbase, &p.ctl->qcnt[slot], v);
}

// Writes the block's buffer to queue[qbase + ...] with one global atomic and
// adds this tile's appends to sm.npush.  Called by all threads of the block.
__device__ __forceinline__ void flush_block(const Params& p, int2* q, Smem& sm, int qbase, int slot) {
    __syncthreads();
    const int n = min(sm.qn, QBUF);
    if (threadIdx.x == 0) {
        sm.npush += sm.qn;
        if (n > 0) sm.qbase = atomicAdd(&p.ctl->qcnt[slot], n);
    }
    __syncthreads();
    if (n > 0) {
        const int b = qbase + sm.qbase;
        for (int k = threadIdx.x; k < n; k += blockDim.x) q[b + k] = sm.qbuf[k];
    }
    if (threadIdx.x == 0) sm.qn = 0;  // the next write to qbuf/qn is behind a __syncthreads
}

// Block-wide exclusive prefix sum of v; returns this thread's offset and puts
// the block total in sm.total.  Contains two __syncthreads.
__device__ __forceinline__ int block_exclusive_scan(int v, Smem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int incl = v;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        int t = __shfl_up_sync(FULL, incl, s);
        if (lane >= s) incl += t;
    }
    if (lane == 31) sm.wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? sm.wsum[lane] : 0;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            int t = __shfl_up_sync(FULL, w, s);
            if (lane >= s) w += t;
        }
        sm.wsum[lane] = w;  // inclusive prefix of warp totals
        if (lane == 31) sm.total = w;
    }
    __syncthreads();
    return (warp > 0 ? sm.wsum[warp - 1] : 0) + incl - v;
}

__device__ __forceinline__ void red_add_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------ grid barrier
// All blocks of a cooperative launch.  Thread 0 of every block adds one
// arrival, a flag (sm.has_ep) and its appended-column count (sm.npush) to the
// arrival word of this barrier with one release reduction (no return value,
// so the block does not wait for the atomic), then polls that same word with
// acquire loads until its arrival count reaches gridDim.x.  The completed
// word carries the level's totals, so every block learns them without a
// separate release store or a counter read: sm.bc_a = appended columns,
// sm.bc_b = blocks that found endpoints.  Words rotate over b % 3; block 0
// clears word (b + 2) % 3 once barrier b is complete (every block has then
// left barrier b - 1, the last user of that word, and none can reach barrier
// b + 2 before block 0 has arrived at b + 1, after the clear).
// If extra_ptr / extra_ptr2 are given, thread 0 also reads them after the
// barrier into sm.bc_c / sm.bc_d.  Returns false (in every thread of the block) when the wait ran
// out of time, the launch deadline passed or a block recorded an error; the
// caller then leaves the kernel.
static __device__ __noinline__ bool grid_sync(Ctl* ctl, int& bid, long long wait_ns,
                                              unsigned long long deadline, Smem& sm,
                                              const int32_t* extra_ptr, const int32_t* extra_ptr2 = nullptr) {
    __syncthreads();
    const int b = bid++;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long inc =
            1ull + ((unsigned long long)(sm.has_ep ? 1 : 0) << 11) + ((unsigned long long)sm.npush << 22);
        unsigned long long* w = &ctl->arrive[b % 3][0];
        red_add_release_u64(w, inc);
        unsigned long long t_end = globaltimer() + (unsigned long long)wait_ns;
        if (t_end > deadline) t_end = deadline;
        unsigned spins = 0;
        unsigned long long v;
        for (;;) {
            v = ld_acquire_u64(w);
            if ((v & 0x7FFull) == (unsigned long long)gridDim.x) break;
            if ((++spins & 15u) == 0) {
                if (ld_volatile(&ctl->err) != 0) { ok = 0; break; }
                if (globaltimer() > t_end) { set_error(ctl, -5 /*BM_ERR_TIMEOUT*/); ok = 0; break; }
            }
        }
        if (blockIdx.x == 0) st_relaxed_u64(&ctl->arrive[(b + 2) % 3][0], 0ull);
        sm.bc_a = (int)((v >> 22) & 0xFFFFFFFFull);
        sm.bc_b = (int)((v >> 11) & 0x7FFull);
        if (extra_ptr) sm.bc_c = ld_volatile(extra_ptr);
        if (extra_ptr2) sm.bc_d = ld_volatile(extra_ptr2);
        sm.npush = 0;
        sm.has_ep = 0;
        sm.ok = ok;
    }
    __syncthreads();
    return sm.ok != 0;
}

struct Counters {  // per-thread, flushed once per launch (32 bits: a thread's share stays far below 2^32)
    unsigned cols, edges, fixes, em, alt;
};

// Adds every thread's v to *dst with one atomic per warp.  Call with the whole
// warp converged (the grid-wide steps below call it once, at their end), so
// that the steps run once per phase do not keep counters live across the
// kernel.
__device__ __forceinline__ void add_to_counter(long long* dst, unsigned v) {
    unsigned long long a = v;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) a += __shfl_down_sync(FULL, a, s);
    if ((threadIdx.x & 31) == 0 && a) atomicAdd((unsigned long long*)dst, a);
}

// ------------------------------------------------------------------ InitBfsArray
// Algorithm 1 InitBfsArray (+ GPUBFS-WR root init, Section 3): level L0 for
// unmatched columns, L0 - 1 for matched ones; root[c] = c for unmatched ones
// (-1 otherwise: 0 is a valid column id).  Unmatched columns with at least one
// row form the first queue segment (a column without rows can never be
// matched, so it is not searched from); all unmatched columns are counted in
// ecnt[slot].  Before that, the column half of FixMatching: a column whose
// row does not point back is unmatched (the row half runs after Alternate).
template <bool WR>
__device__ __forceinline__ void step_init(const Params& p, int2* q, int slot, Counters& cnt, Smem& sm) {
    const int nc = p.nc;
    int nfree = 0, niso = 0;
    unsigned fixes = 0;
    // 4 columns per thread per pass, their loads in flight together (a pass appends at
    // most 4 x blockDim <= QBUF entries per block)
    const int T = blockDim.x;
    for (int base = blockIdx.x * 4 * T; base < nc; base += gridDim.x * 4 * T) {  // block-uniform
        int c[4], r[4], back[4], deg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = base + u * T + threadIdx.x;
            r[u] = c[u] < nc ? __ldcg(&p.cmatch[c[u]]) : -2;
            if (r[u] >= 0 && !idx_ok(p, r[u], p.nr)) r[u] = -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            back[u] = r[u] >= 0 ? __ldcg(&p.rmatch[r[u]]) : -1;
            deg[u] = c[u] < nc ? __ldg(&p.col_ptr[c[u] + 1]) - __ldg(&p.col_ptr[c[u]]) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= nc) continue;
            if (r[u] >= 0 && back[u] != c[u]) {
                __stcg(&p.cmatch[c[u]], -1);
                r[u] = -1;
                ++fixes;
            }
            const bool is_free = (r[u] < 0);
            __stcg(&p.level[c[u]], is_free ? L0 : L0 - 1);
            if (WR) __stcg(&p.root[c[u]], is_free ? c[u] : -1);
            if (is_free) {
                if (p.crec) __stcg(&p.crec[c[u]], make_int2(-1, -1));
                ++nfree;
                if (deg[u] > 0) push_block(p, q, sm, 0, slot, make_int2(c[u], c[u]));
                else ++niso;
            }
        }
        flush_block(p, q, sm, 0, slot);
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        nfree += __shfl_down_sync(FULL, nfree, s);
        niso += __shfl_down_sync(FULL, niso, s);
    }
    if ((threadIdx.x & 31) == 0 && nfree) atomicAdd(&p.ctl->ecnt[slot], nfree);
    if ((threadIdx.x & 31) == 0 && niso) atomicAdd(&p.ctl->icnt[slot], niso);
    add_to_counter(&p.ctl->fix_repairs, fixes);
}

// Between phases in the one-endpoint GPUBFS-WR mode (where Alternate's walks
// cannot meet, so FixMatching has nothing to repair and the columns not
// touched by the search keep their InitBfsArray values): the columns the
// search inserted go back to "unvisited" and the roots that are still
// unmatched are appended to the other queue buffer as the next phase's roots.
// DET (deterministic option): the inserted columns' tree-entry keys and the
// roots' endpoint picks (the roots' own key words) go back to "none" too.
// SERVED: a root counts as matched when its level slot says it took an
// endpoint (-(row)), not by its cmatch entry -- the same set once Alternate
// has walked every path to its root, and known before: this pass may then
// run while the walks are still going (neither touches what the other reads
// or writes: the walks use crec, pred, cmatch and rmatch; this pass the
// queue, level, root and the keys).
template <bool WR, bool DET = false, bool SERVED = false>
__device__ __forceinline__ void step_next_roots(const Params& p, const int2* q, int n_roots, int tail,
                                                int2* q_next, int slot, Smem& sm) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    // 4 entries per thread per pass, their loads in flight together
    for (int i0 = n_roots + tid; i0 < tail; i0 += 4 * nthr) {
        int c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = i0 + u * nthr < tail ? __ldcg(&q[i0 + u * nthr]).x : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] < 0 || !idx_ok(p, c[u], p.nc)) continue;
            __stcg(&p.level[c[u]], L0 - 1);
            if (WR) __stcg(&p.root[c[u]], -1);
            if (DET) __stcg(&p.dkey[c[u]], ~0ull);
        }
    }
    const int T = blockDim.x;
    for (int base = blockIdx.x * T * 4; base < n_roots; base += gridDim.x * T * 4) {  // block-uniform
        int c[4], m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + u * T + threadIdx.x;
            c[u] = i < n_roots ? __ldcg(&q[i]).x : -1;
            if (c[u] >= 0 && !idx_ok(p, c[u], p.nc)) c[u] = -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            m[u] = c[u] < 0 ? 0 : SERVED ? (__ldcg(&p.level[c[u]]) == L0 ? -1 : 0) : __ldcg(&p.cmatch[c[u]]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] < 0) continue;
            if (DET) __stcg(&p.dkey[c[u]], ~0ull);
            if (m[u] < 0) {
                push_block(p, q_next, sm, 0, slot, make_int2(c[u], c[u]));
            } else {
                __stcg(&p.level[c[u]], L0 - 1);
                if (WR) __stcg(&p.root[c[u]], -1);
            }
        }
    }
    flush_block(p, q_next, sm, 0, slot);  // a full buffer spills to global appends meanwhile
}

// ------------------------------------------------------------------ BFS level
// Loads tile entries [qb + first, qb + first + tw) of the queue (one per
// thread; threads >= tw idle) and lays the tile's adjacency out in shared
// memory: sm.off (exclusive prefix of degrees), sm.beg, sm.col, sm.root,
// sm.total.  The queue entry carries the root, so the column's row range and
// the GPUBFS-WR root test (Algorithm 4: skip the column if its root is already
// served) are two independent loads whose latency overlaps the prefix sum; a
// column whose root is served keeps its place in the prefix sum but gets
// sm.col = -1 and its edges are skipped.  If tile_ctr is given, thread 0 also
// takes the block's next work item from it: sm.tile = ctr_base + the counter's
// old value, after adding `grab` (a tile index with grab 1 and ctr_base
// gridDim.x; a queue position with a range width and the end of the static
// ranges in the guided schedule).  Ends with __syncthreads.
template <bool WR, bool NC = true>
__device__ __forceinline__ void tile_load(const Params& p, const int2* queue, int qb, int q, int first, int tw,
                                          Smem& sm, Counters& cnt, int32_t* tile_ctr, int grab = 1, int ctr_base = -1) {
    const int t = threadIdx.x;
    const int i = first + t;
    int c = -1, beg = 0, deg = 0, myroot = -1, rlev = L0;
    if (t < tw && i < q) {
        const int2 ent = __ldcg(&queue[qb + i]);
        c = ent.x;
        myroot = ent.y;
        if (!idx_ok(p, c, p.nc) || (WR && !idx_ok(p, myroot, p.nc))) {  // checked build only
            c = -1;
        } else {
            beg = ld_csr<NC>(&p.col_ptr[c]);
            deg = ld_csr<NC>(&p.col_ptr[c + 1]) - beg;
            if (WR) rlev = __ldcg(&p.level[myroot]);
        }
    }
    if (t == 0 && tile_ctr) sm.tile = (ctr_base < 0 ? (int)gridDim.x : ctr_base) + atomicAdd(tile_ctr, grab);
    const int off = block_exclusive_scan(deg, sm);
    if (WR && rlev < L0 - 1) c = -1;  // Algorithm 4: root already served
    if (c >= 0) cnt.cols++;
    sm.off[t] = off;
    sm.beg[t] = beg;
    sm.col[t] = c;
    sm.root[t] = myroot;
    __syncthreads();
}

// tile_load for tiles of 2 x blockDim entries (two per thread; 2 x blockDim
// <= MAX_BLOCK): the one-block-per-graph routine, where a level's tiles run
// one after another in one block, gets twice the columns (and their loads)
// in flight per tile.  Ends with __syncthreads.
template <bool WR, bool NC = true>
__device__ __forceinline__ void tile_load2(const Params& p, const int2* queue, int qb, int q, int first, Smem& sm,
                                           Counters& cnt) {
    const int t = threadIdx.x;
    int c[2], beg[2], deg[2], rt[2], rl[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int i = first + 2 * t + u;
        c[u] = -1; beg[u] = 0; deg[u] = 0; rt[u] = -1; rl[u] = L0;
        if (i < q) {
            const int2 ent = __ldcg(&queue[qb + i]);
            c[u] = ent.x;
            rt[u] = ent.y;
            if (!idx_ok(p, c[u], p.nc) || (WR && !idx_ok(p, rt[u], p.nc))) c[u] = -1;
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (c[u] >= 0) {
            beg[u] = ld_csr<NC>(&p.col_ptr[c[u]]);
            deg[u] = ld_csr<NC>(&p.col_ptr[c[u] + 1]) - beg[u];
            if (WR) rl[u] = __ldcg(&p.level[rt[u]]);
        }
    }
    const int off = block_exclusive_scan(deg[0] + deg[1], sm);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (WR && rl[u] < L0 - 1) c[u] = -1;  // Algorithm 4: root already served
        if (c[u] >= 0) cnt.cols++;
        sm.off[2 * t + u] = off + (u ? deg[0] : 0);
        sm.beg[2 * t + u] = beg[u];
        sm.col[2 * t + u] = c[u];
        sm.root[2 * t + u] = rt[u];
    }
    __syncthreads();
}

// Visits every edge of the loaded tile (Algorithm 2 / 4 loop body), ILP edges
// per thread with their loads in flight together.  push_col(cm) appends a
// column inserted at level lvl + 1, push_end(r) an endpoint row.
// direct: claim with the atomic alone (small frontiers: saves a dependent load);
// otherwise test first and claim only unvisited columns.  RV (row stamps
// p.rvis available): use_rv claims through the row stamps with `stamp` (see
// the header comment); otherwise claims go to the column's level entry and,
// with RV, the winner also stamps the row.
// CA: the matched column of a row (rmatch) and the column's level are read
// through L1.  Only for the grid-wide kernel, where every level starts after
// the grid barrier's acquire (which makes these loads see the previous
// levels' and phases' writes): within a level a matched row's column does not
// change, and a stale "unvisited" level only costs a failed claim.
template <bool WR, class PushCol, class PushEnd, bool NC = true, bool RV = false, bool CA = false>
__device__ __forceinline__ void tile_edges(const Params& p, int tw, int lvl, bool direct, Smem& sm,
                                           Counters& cnt, PushCol push_col, PushEnd push_end, int stamp = 0,
                                           bool use_rv = false) {
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int total = sm.total;
    for (int e0 = 0; e0 < total; e0 += T * ILP) {
        int own[ILP], r[ILP], cm[ILP], lv[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const int e = e0 + u * T + t;
            own[u] = -1;
            r[u] = -1;
            if (e < total) {
                int lo = 0, hi = tw - 1;  // last k with off[k] <= e
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sm.off[mid] <= e) lo = mid; else hi = mid - 1;
                }
                if (sm.col[lo] >= 0) {
                    own[u] = lo;
                    r[u] = ld_csr<NC>(&p.row_idx[sm.beg[lo] + (e - sm.off[lo])]);
                    if (!idx_ok(p, r[u], p.nr)) own[u] = r[u] = -1;
                }
            }
        }
        if (RV && use_rv) {
            // rmatch[r] and the claim of the row: independent, in flight together
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                cm[u] = -3;
                lv[u] = stamp;
                if (own[u] >= 0) {
                    cm[u] = CA ? __ldca(&p.rmatch[r[u]]) : __ldcg(&p.rmatch[r[u]]);
                    lv[u] = atomicMax(&p.rvis[r[u]], stamp);
                }
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (cm[u] >= 0 && !idx_ok(p, cm[u], p.nc)) cm[u] = -3;  // checked build only
        } else {
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                cm[u] = (own[u] >= 0) ? (CA ? __ldca(&p.rmatch[r[u]]) : __ldcg(&p.rmatch[r[u]])) : -3;
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (cm[u] >= 0 && !idx_ok(p, cm[u], p.nc)) cm[u] = -3;  // checked build only
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                lv[u] = (cm[u] < 0 || direct) ? L0 - 1
                                                    : (CA ? __ldca(&p.level[cm[u]]) : __ldcg(&p.level[cm[u]]));
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (own[u] < 0) continue;
            const int col = sm.col[own[u]];
            const int rt = sm.root[own[u]];
            cnt.edges++;
            if (cm[u] >= 0) {
                cnt.em++;
                // matched row: its column joins the next level unless already reached
                bool won;
                if (RV && use_rv) won = lv[u] < stamp;
                else won = lv[u] == L0 - 1 && atomicCAS(&p.level[cm[u]], L0 - 1, lvl + 1) == L0 - 1;
                if (won) {
                    if (RV) {
                        if (use_rv) __stcg(&p.level[cm[u]], lvl + 1);
                        else __stcg(&p.rvis[r[u]], stamp);
                    }
                    __stcg(&p.pred[r[u]], col);
                    if (WR) __stcg(&p.root[cm[u]], rt);
                    if (RV) __stcg(&p.crec[cm[u]], make_int2(col, r[u]));
                    push_col(make_int2(cm[u], rt));
                }
            } else if (cm[u] == -1) {
                // unmatched row: an augmenting path ends here
                const int row = r[u];
                if (WR && p.one_ep) {
                    if (__ldcg(&p.level[rt]) == L0 && atomicCAS(&p.rmatch[row], -1, -2) == -1) {
                        if (atomicCAS(&p.level[rt], L0, -row) == L0) {
                            __stcg(&p.pred[row], col);
                            push_end(row);
                            sm.has_ep = 1;
                        } else {
                            atomicExch(&p.rmatch[row], -1);  // root served meanwhile: give the row back
                        }
                    }
                } else if (atomicCAS(&p.rmatch[row], -1, -2) == -1) {
                    if (WR) __stcg(&p.level[rt], L0 - 2);
                    __stcg(&p.pred[row], col);
                    push_end(row);
                    sm.has_ep = 1;
                }
            }
        }
    }
}

// Visits edge (col, r) of a column of root rt, r's match being cm, in the
// one-block-per-graph routine with shared-memory marks (SB): a matched row's
// column joins the next level if its bit in p.vis was clear (Algorithm 2); an
// unmatched row ends an augmenting path if the root's bit in p.srv was clear
// (Algorithm 4, one endpoint per root), the row held by the -2 mark meanwhile.
template <class PushCol, class PushEnd>
__device__ __forceinline__ void sb_visit(const Params& p, int col, int rt, int r, int cm, Counters& cnt,
                                         PushCol push_col, PushEnd push_end) {
    cnt.edges++;
    if (cm >= 0) {
        cnt.em++;
        if (!sb_test(p.vis, cm) && sb_claim(p.vis, cm)) {
            __stcg(&p.pred[r], col);
            push_col(make_int2(cm, rt));
        }
    } else if (cm == -1) {
        if (!sb_test(p.srv, rt) && atomicCAS(&p.rmatch[r], -1, -2) == -1) {
            if (sb_claim(p.srv, rt)) {
                __stcg(&p.pred[r], col);
                push_end(r);
            } else {
                atomicExch(&p.rmatch[r], -1);  // root served meanwhile: give the row back
            }
        }
    }
}

// One BFS level of the one-block-per-graph routine with its tree and served-root
// marks in the shared-memory bitmaps (SB): the columns of queue positions
// [qb, qb + q), at level lvl, are expanded by warps, each taking 32 queue
// entries at a time from the counter *grab (zeroed before the level).  A warp
// scans its columns' degrees with shuffles and visits their edges 32 x ILP at
// a time; the column owning edge j is found from which of the warp's columns
// start at or before j (one OR-reduction of the start positions per 32 edges
// and a population count per lane), so no per-edge search and no block-wide
// scan or barrier per tile are needed.  Edges are visited by sb_visit.
// Columns whose root is already served are skipped whole.  A column of more
// than HUB_DEG edges is set aside in sm.hub (up to HUB_MAX a level, counted
// in *nhub) for block_hubs_sb, so that one warp does not walk it alone.  The
// warp's compacted column records use its 32 slots of sm.beg / sm.col / sm.root.
template <bool NC, bool CA, class PushCol, class PushEnd>
__device__ __forceinline__ void warp_expand_sb(const Params& p, int qb, int q, int* grab, int* nhub, Smem& sm,
                                               Counters& cnt, PushCol push_col, PushEnd push_end) {
    const int lane = threadIdx.x & 31;
    const int wb = threadIdx.x & ~31;
    int* const s_base = &sm.beg[wb];  // beg - start: row_idx position = s_base[k] + j
    int* const s_col = &sm.col[wb];
    int* const s_root = &sm.root[wb];
    int g = 0;
    if (lane == 0) g = atomicAdd(grab, 32);
    g = __shfl_sync(FULL, g, 0);
    int2 ent = make_int2(-1, -1);
    if (g + lane < q) ent = __ldcg(&p.queue[qb + g + lane]);
    for (;;) {
        if (g >= q) break;
        int c = -1, rt = -1, beg = 0, deg = 0;
        const bool mine = g + lane < q;
        const int2 cur = ent;
        // the next group's queue entries are loaded while this group is expanded
        int g2 = 0;
        if (lane == 0) g2 = atomicAdd(grab, 32);
        g2 = __shfl_sync(FULL, g2, 0);
        ent = make_int2(-1, -1);
        if (g2 + lane < q) ent = __ldcg(&p.queue[qb + g2 + lane]);
        if (mine) {
            c = cur.x;
            rt = cur.y;
            if (!idx_ok(p, c, p.nc) || !idx_ok(p, rt, p.nc)) {  // checked build only
                c = -1;
            } else {
                beg = ld_csr<NC>(&p.col_ptr[c]);
                deg = ld_csr<NC>(&p.col_ptr[c + 1]) - beg;
                if (sb_test(p.srv, rt)) c = -1;  // Algorithm 4: root already served
            }
        }
        if (c < 0) deg = 0;
        else cnt.cols++;
        if (deg > HUB_DEG) {  // the whole block takes it after the warps
            const int h = atomicAdd(nhub, 1);
            if (h < HUB_MAX) {
                sm.hub[0][h] = c;
                sm.hub[1][h] = rt;
                sm.hub[2][h] = beg;
                sm.hub[3][h] = deg;
                deg = 0;
            }
        }
        int incl = deg;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int start = incl - deg;
        const int rank = __popc(__ballot_sync(FULL, deg > 0) & ((1u << lane) - 1));
        __syncwarp();  // the previous group's reads of the slots are done
        if (deg > 0) {
            s_base[rank] = beg - start;
            s_col[rank] = c;
            s_root[rank] = rt;
        }
        __syncwarp();
        int before = 0;  // columns with edges that start before the current 32 edges
        for (int j0 = 0; j0 < total; j0 += 32 * ILP) {
            int own[ILP], r[ILP], cm[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                const int J0 = j0 + 32 * u;  // warp-uniform
                const unsigned starts =
                    __reduce_or_sync(FULL, (deg > 0 && start >= J0 && start < J0 + 32) ? 1u << (start - J0) : 0u);
                const int j = J0 + lane;
                own[u] = -1;
                r[u] = -1;
                if (j < total) {
                    const int k = before + __popc(starts & (0xFFFFFFFFu >> (31 - lane))) - 1;
                    own[u] = k;
                    r[u] = ld_csr<NC>(&p.row_idx[s_base[k] + j]);
                    if (!idx_ok(p, r[u], p.nr)) own[u] = r[u] = -1;
                }
                before += __popc(starts);
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                cm[u] = (own[u] >= 0) ? (CA ? __ldca(&p.rmatch[r[u]]) : __ldcg(&p.rmatch[r[u]])) : -3;
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (cm[u] >= 0 && !idx_ok(p, cm[u], p.nc)) cm[u] = -3;  // checked build only
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (own[u] >= 0) sb_visit(p, s_col[own[u]], s_root[own[u]], r[u], cm[u], cnt, push_col, push_end);
        }
        g = g2;
    }
}

// The columns warp_expand_sb set aside (n of them, n <= HUB_MAX), one after
// another by the whole block, ILP edges per thread in flight.  A column whose
// root was served since it was set aside is skipped (Algorithm 4).
template <bool NC, bool CA, class PushCol, class PushEnd>
__device__ __forceinline__ void block_hubs_sb(const Params& p, int n, Smem& sm, Counters& cnt, PushCol push_col,
                                              PushEnd push_end) {
    const int T = blockDim.x, t = threadIdx.x;
    for (int h = 0; h < n; ++h) {
        const int col = sm.hub[0][h], rt = sm.hub[1][h], beg = sm.hub[2][h], deg = sm.hub[3][h];
        for (int e0 = 0; e0 < deg; e0 += T * ILP) {
            if (sb_test(p.srv, rt)) break;  // no barrier in this loop: a thread may leave alone
            int r[ILP], cm[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                const int e = e0 + u * T + t;
                r[u] = e < deg ? ld_csr<NC>(&p.row_idx[beg + e]) : -1;
                if (r[u] >= 0 && !idx_ok(p, r[u], p.nr)) r[u] = -1;
            }
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                cm[u] = r[u] >= 0 ? (CA ? __ldca(&p.rmatch[r[u]]) : __ldcg(&p.rmatch[r[u]])) : -3;
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (cm[u] >= 0 && !idx_ok(p, cm[u], p.nc)) cm[u] = -3;  // checked build only
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (r[u] >= 0) sb_visit(p, col, rt, r[u], cm[u], cnt, push_col, push_end);
        }
    }
}

// warp_expand_sb's walk for any claim rule (the deterministic option's block
// routine): the columns of queue positions [qb, qb + q) are expanded by warps, each taking 32 queue
// entries at a time from the counter *grab (zeroed before the level) and
// loading the next group's entries while it expands the current one.
// entry(e, c, rt, beg, deg) completes a queue entry into its column, root and
// row range (c = -1: the column is skipped, e.g. its root is served).  A warp
// scans its columns' degrees with shuffles and hands their edges out 32 x ILP
// at a time: the column owning edge j is the last one starting at or before j,
// found from one OR-reduction of the start positions per 32 edges and a
// population count per lane, so there is no per-edge search and no block-wide
// scan or barrier per tile.  round(own, r, s_col, s_root) visits up to ILP
// edges of the thread (row r[u] of the column s_col[own[u]] of root
// s_root[own[u]]; own[u] < 0: none).  A column of more than HUB_DEG edges is
// set aside in sm.hub (up to HUB_MAX a level, counted in *nhub) for
// block_hubs, so that one warp does not walk it alone.  The warp's compacted
// column records use its 32 slots of sm.beg / sm.col / sm.root.
template <bool NC, class Entry, class Round>
__device__ __forceinline__ void warp_expand(const Params& p, int qb, int q, int* grab, int* nhub, Smem& sm,
                                            Counters& cnt, Entry entry, Round round) {
    const int lane = threadIdx.x & 31;
    const int wb = threadIdx.x & ~31;
    int* const s_base = &sm.beg[wb];  // beg - start: row_idx position = s_base[k] + j
    int* const s_col = &sm.col[wb];
    int* const s_root = &sm.root[wb];
    int g = 0;
    if (lane == 0) g = atomicAdd(grab, 32);
    g = __shfl_sync(FULL, g, 0);
    int2 ent = make_int2(-1, -1);
    if (g + lane < q) ent = __ldcg(&p.queue[qb + g + lane]);
    for (;;) {
        if (g >= q) break;
        int c = -1, rt = -1, beg = 0, deg = 0;
        const bool mine = g + lane < q;
        const int2 cur = ent;
        // the next group's queue entries are loaded while this group is expanded
        int g2 = 0;
        if (lane == 0) g2 = atomicAdd(grab, 32);
        g2 = __shfl_sync(FULL, g2, 0);
        ent = make_int2(-1, -1);
        if (g2 + lane < q) ent = __ldcg(&p.queue[qb + g2 + lane]);
        if (mine) entry(cur, c, rt, beg, deg);
        if (c < 0) deg = 0;
        else cnt.cols++;
        if (deg > HUB_DEG) {  // the whole block takes it after the warps
            const int h = atomicAdd(nhub, 1);
            if (h < HUB_MAX) {
                sm.hub[0][h] = c;
                sm.hub[1][h] = rt;
                sm.hub[2][h] = beg;
                sm.hub[3][h] = deg;
                deg = 0;
            }
        }
        int incl = deg;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int start = incl - deg;
        const int rank = __popc(__ballot_sync(FULL, deg > 0) & ((1u << lane) - 1));
        __syncwarp();  // the previous group's reads of the slots are done
        if (deg > 0) {
            s_base[rank] = beg - start;
            s_col[rank] = c;
            s_root[rank] = rt;
        }
        __syncwarp();
        int before = 0;  // columns with edges that start before the current 32 edges
        for (int j0 = 0; j0 < total; j0 += 32 * ILP) {
            int own[ILP], r[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                const int J0 = j0 + 32 * u;  // warp-uniform
                const unsigned starts =
                    __reduce_or_sync(FULL, (deg > 0 && start >= J0 && start < J0 + 32) ? 1u << (start - J0) : 0u);
                const int j = J0 + lane;
                own[u] = -1;
                r[u] = -1;
                if (j < total) {
                    const int k = before + __popc(starts & (0xFFFFFFFFu >> (31 - lane))) - 1;
                    own[u] = k;
                    r[u] = ld_csr<NC>(&p.row_idx[s_base[k] + j]);
                    if (!idx_ok(p, r[u], p.nr)) own[u] = r[u] = -1;
                }
                before += __popc(starts);
            }
            round(own, r, s_col, s_root);
        }
        g = g2;
    }
}

// The columns warp_expand set aside (n of them, n <= HUB_MAX), one after
// another by the whole block, ILP edges per thread in flight; the same
// round(own, r, s_col, s_root) visits them.  A thread stops a column once
// alive(root) is false (its root served since it was set aside: Algorithm 4).
template <bool NC, class Alive, class Round>
__device__ __forceinline__ void block_hubs(const Params& p, int n, Smem& sm, Alive alive, Round round) {
    const int T = blockDim.x, t = threadIdx.x;
    for (int h = 0; h < n; ++h) {
        const int rt = sm.hub[1][h], beg = sm.hub[2][h], deg = sm.hub[3][h];
        for (int e0 = 0; e0 < deg; e0 += T * ILP) {
            if (!alive(rt)) break;  // no barrier in this loop: a thread may leave alone
            int own[ILP], r[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                const int e = e0 + u * T + t;
                r[u] = e < deg ? ld_csr<NC>(&p.row_idx[beg + e]) : -1;
                if (r[u] >= 0 && !idx_ok(p, r[u], p.nr)) r[u] = -1;
                own[u] = r[u] >= 0 ? 0 : -1;
            }
            round(own, r, &sm.hub[0][h], &sm.hub[1][h]);
        }
    }
}

// Expands the queue segment [qb, qe) whose columns are at level lvl, over the
// whole grid.  New columns are appended at qe + (slot count), endpoints at
// ep_phase (the phase's running count).  Frontiers of at most one tile per
// block (the deep, narrow levels of long augmenting paths) take their tile
// from blockIdx.x alone and claim columns by CAS without a test load.  GRID:
// called by the persistent kernel between grid barriers (L1 reads, see
// tile_edges; wider levels are handed out in guided ranges, below); the
// per-step kernels of the host-driven loop leave it off and take fixed tiles
// from the step's tile counter.
template <bool WR, bool RV = false, bool GRID = false>
__device__ __forceinline__ void step_expand(const Params& p, int2* queue, int qb, int qe, int lvl, int slot,
                                            Counters& cnt, Smem& sm, int stamp = 0, int32_t* ep_ctr = nullptr) {
    const int q = qe - qb;
    // tile width: spread small frontiers over many blocks, never above blockDim
    int tw = (q + gridDim.x - 1) / gridDim.x;
    tw = (tw + 31) & ~31;
    if (tw > (int)blockDim.x) tw = blockDim.x;
    if (tw < 32) tw = 32;
    const int ntiles = (q + tw - 1) / tw;
    const bool narrow = ntiles <= (int)gridDim.x;
    auto push_col = [&](int2 v) { push_block(p, queue, sm, qe, slot, v); };
    int32_t* const epc = ep_ctr ? ep_ctr : &p.ctl->ep_phase;
    auto push_end = [&](int v) { push(p.endpoints, 0, epc, v); };
    if (GRID && !narrow) {
        // Guided self-scheduling of a wide level: block b first takes columns
        // [b w0, (b + 1) w0) with w0 ~ q / 2G, then ranges from a position
        // counter, each about 1/2G of what is left past its current range (32
        // to blockDim columns), prefetched while it works on the current one:
        // large ranges first, small ones at the end, so that no block is left
        // with a heavy 512-column tile when the others are done.
        const int G = gridDim.x, T = blockDim.x;
        auto clamp_w = [&](long long w) { return (int)min((long long)T, max(32LL, (w + 31) & ~31LL)); };
        const int w0 = clamp_w(((long long)q + 2 * G - 1) / (2 * G));
        int first = (int)min((long long)blockIdx.x * w0, (long long)q);
        int width = w0;
        while (first < q) {  // block-uniform
            const int grab = clamp_w(((long long)q - first - width) / (2 * G));
            tile_load<WR>(p, queue, qb, q, first, width, sm, cnt, &p.ctl->tcnt[slot], grab, G * w0);
            const int next_first = sm.tile;
            tile_edges<WR, decltype(push_col), decltype(push_end), true, RV, GRID>(p, width, lvl, false, sm, cnt,
                                                                                    push_col, push_end, stamp,
                                                                                    q <= RV_MAX_Q);
            flush_block(p, queue, sm, qe, slot);
            first = next_first;
            width = grab;
        }
        return;
    }
    for (int tile = blockIdx.x; tile < ntiles;) {  // block-uniform
        tile_load<WR>(p, queue, qb, q, tile * tw, tw, sm, cnt, narrow ? nullptr : &p.ctl->tcnt[slot]);
        const int next_tile = narrow ? ntiles : sm.tile;
        tile_edges<WR, decltype(push_col), decltype(push_end), true, RV, GRID>(p, tw, lvl, narrow, sm, cnt,
                                                                                push_col, push_end, stamp,
                                                                                q <= RV_MAX_Q);
        flush_block(p, queue, sm, qe, slot);
        tile = next_tile;
    }
}

// ------------------------------------------------------------------ deterministic option
// The level step with every choice that the code above leaves to whichever
// thread comes first fixed by a smallest-id rule, one level at a time (the
// level-synchronous reading of Algorithm 4 with one endpoint per root):
//  * Tree entry: dkey[c] holds (level << 32 | parent) once column c is in a
//    tree, all ones before.  A level-L column that reaches c through c's
//    matched row takes atomicMin((L + 1) << 32 | itself): an entry from an
//    earlier level is never replaced, and of the level-L parents the smallest
//    wins.  The claimer that found the word empty appends c; when the next
//    level loads c it reads the winner and fills in c's root (the parent's),
//    level, pred and crec.
//  * Endpoints: an unmatched row that no root owns keeps, in ekey[r], the
//    smallest (root << 32 | column) that reaches it during the level; its
//    first offerer lists it in ecand.  After the level's barrier every listed
//    row offers itself to its root (atomicMin of the row id in the root's own
//    dkey word: roots are unmatched, so no claim ever touches it); after one
//    more barrier each root takes the smallest row that offered itself
//    (rmatch[r] = -2, pred[r] = the column, level[root] = -(row)); the other
//    rows stay unmatched and their offers are cleared.
//  * A root that took an endpoint at level L stops at level L + 1; the
//    columns it claimed for level L + 1 stay claimed.
// The matching and every counter are then the same for every run and launch
// geometry.
constexpr unsigned long long DKEY_NONE = ~0ull;

// tile_load for the deterministic option: entries of levels after L0 carry
// no root yet (-1); each is completed here from its tree-entry word before
// the GPUBFS-WR root test.  Ends with __syncthreads.
template <bool NC = true>
__device__ __forceinline__ void tile_load_det(const Params& p, const int2* queue, int qb, int q, int first, int tw,
                                              int lvl, Smem& sm, Counters& cnt, int32_t* tile_ctr, int grab = 1,
                                              int ctr_base = -1) {
    const int t = threadIdx.x;
    const int i = first + t;
    int c = -1, beg = 0, deg = 0, myroot = -1, rlev = L0;
    if (t < tw && i < q) {
        const int2 ent = __ldcg(&queue[qb + i]);
        c = ent.x;
        if (!idx_ok(p, c, p.nc)) {  // checked build only
            c = -1;
        } else {
            beg = ld_csr<NC>(&p.col_ptr[c]);
            deg = ld_csr<NC>(&p.col_ptr[c + 1]) - beg;
            if (lvl == L0) {
                myroot = ent.y;  // a root: (c, c)
            } else {
                const unsigned long long k = __ldcg(&p.dkey[c]);
                const int par = (int)(unsigned)(k & 0xffffffffull);
                const int row = __ldcg(&p.cmatch[c]);
                if (!idx_ok(p, par, p.nc) || !idx_ok(p, row, p.nr)) {
                    c = -1;
                } else {
                    myroot = __ldcg(&p.root[par]);
                    __stcg(&p.root[c], myroot);
                    __stcg(&p.level[c], lvl);
                    __stcg(&p.pred[row], par);
                    if (p.crec) __stcg(&p.crec[c], make_int2(par, row));
                }
            }
            if (c >= 0 && !idx_ok(p, myroot, p.nc)) c = -1;
            if (c >= 0) rlev = __ldcg(&p.level[myroot]);
        }
    }
    if (t == 0 && tile_ctr) sm.tile = (ctr_base < 0 ? (int)gridDim.x : ctr_base) + atomicAdd(tile_ctr, grab);
    const int off = block_exclusive_scan(c >= 0 ? deg : 0, sm);
    if (rlev < L0 - 1) c = -1;  // Algorithm 4: root already served
    if (c >= 0) cnt.cols++;
    sm.off[t] = off;
    sm.beg[t] = beg;
    sm.col[t] = c;
    sm.root[t] = myroot;
    __syncthreads();
}

// tile_edges for the deterministic option (the rules above); lvl is the level
// of the tile's columns; push_off(r) lists a row that received its first
// offer of the level in ecand.
template <class PushCol, class PushOff, bool NC = true>
__device__ __forceinline__ void tile_edges_det(const Params& p, int tw, int lvl, Smem& sm, Counters& cnt,
                                               PushCol push_col, PushOff push_off) {
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int total = sm.total;
    const unsigned long long next_lv = (unsigned long long)(unsigned)(lvl + 1) << 32;
    for (int e0 = 0; e0 < total; e0 += T * ILP) {
        int own[ILP], r[ILP], cm[ILP];
        unsigned long long key[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const int e = e0 + u * T + t;
            own[u] = -1;
            r[u] = -1;
            if (e < total) {
                int lo = 0, hi = tw - 1;  // last k with off[k] <= e
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sm.off[mid] <= e) lo = mid; else hi = mid - 1;
                }
                if (sm.col[lo] >= 0) {
                    own[u] = lo;
                    r[u] = ld_csr<NC>(&p.row_idx[sm.beg[lo] + (e - sm.off[lo])]);
                    if (!idx_ok(p, r[u], p.nr)) own[u] = r[u] = -1;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) cm[u] = own[u] >= 0 ? __ldcg(&p.rmatch[r[u]]) : -3;
#pragma unroll
        for (int u = 0; u < ILP; ++u)
            if (cm[u] >= 0 && !idx_ok(p, cm[u], p.nc)) cm[u] = -3;  // checked build only
#pragma unroll
        for (int u = 0; u < ILP; ++u)
            key[u] = cm[u] < 0 ? 0ull : __ldcg(&p.dkey[cm[u]]);
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (own[u] < 0) continue;
            const int col = sm.col[own[u]];
            cnt.edges++;
            if (cm[u] >= 0) {
                cnt.em++;
                // keys only decrease: a stale key that is not above ours is final
                const unsigned long long want = next_lv | (unsigned)col;
                if (key[u] > want && atomicMin(&p.dkey[cm[u]], want) == DKEY_NONE) push_col(make_int2(cm[u], -1));
            } else if (cm[u] == -1) {
                const unsigned long long want =
                    ((unsigned long long)(unsigned)sm.root[own[u]] << 32) | (unsigned)col;
                if (atomicMin(&p.ekey[r[u]], want) == DKEY_NONE) push_off(r[u]);
                sm.has_ep = 1;
            }
        }
    }
}

// step_expand for the deterministic option (same schedule: guided ranges on
// wide levels, one static tile per block on narrow ones).
__device__ __forceinline__ void step_expand_det(const Params& p, int2* queue, int qb, int qe, int lvl, int slot,
                                                Counters& cnt, Smem& sm) {
    const int q = qe - qb;
    int tw = (q + gridDim.x - 1) / gridDim.x;
    tw = (tw + 31) & ~31;
    if (tw > (int)blockDim.x) tw = blockDim.x;
    if (tw < 32) tw = 32;
    const int ntiles = (q + tw - 1) / tw;
    const bool narrow = ntiles <= (int)gridDim.x;
    auto push_col = [&](int2 v) { push_block(p, queue, sm, qe, slot, v); };
    auto push_off = [&](int r) { push(p.ecand, 0, &p.ctl->dcnt[slot], r); };
    if (!narrow) {
        const int G = gridDim.x, T = blockDim.x;
        auto clamp_w = [&](long long w) { return (int)min((long long)T, max(32LL, (w + 31) & ~31LL)); };
        const int w0 = clamp_w(((long long)q + 2 * G - 1) / (2 * G));
        int first = (int)min((long long)blockIdx.x * w0, (long long)q);
        int width = w0;
        while (first < q) {  // block-uniform
            const int grab = clamp_w(((long long)q - first - width) / (2 * G));
            tile_load_det(p, queue, qb, q, first, width, lvl, sm, cnt, &p.ctl->tcnt[slot], grab, G * w0);
            const int next_first = sm.tile;
            tile_edges_det(p, width, lvl, sm, cnt, push_col, push_off);
            flush_block(p, queue, sm, qe, slot);
            first = next_first;
            width = grab;
        }
        return;
    }
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {  // block-uniform
        tile_load_det(p, queue, qb, q, tile * tw, tw, lvl, sm, cnt, nullptr);
        tile_edges_det(p, tw, lvl, sm, cnt, push_col, push_off);
        flush_block(p, queue, sm, qe, slot);
    }
}

// After a level with offers (n rows listed in ecand): every listed row
// offers itself to the root that won it.  Entries i0, i0 + stride, ... (the
// grid, or one block).
__device__ __forceinline__ void det_offer(const Params& p, int n, int i0, int stride) {
    for (int i = i0; i < n; i += stride) {
        const int r = __ldcg(&p.ecand[i]);
        if (!idx_ok(p, r, p.nr)) continue;
        const int rho = (int)(__ldcg(&p.ekey[r]) >> 32);
        if (!idx_ok(p, rho, p.nc)) continue;
        atomicMin(&p.dkey[rho], (unsigned long long)(unsigned)r);
    }
}

// Then every root takes the smallest row that offered itself as its one
// endpoint (push_end appends it to the endpoint list); every listed row's
// offer is cleared.
template <class PushEnd>
__device__ __forceinline__ void det_take(const Params& p, int n, int i0, int stride, PushEnd push_end) {
    for (int i = i0; i < n; i += stride) {
        const int r = __ldcg(&p.ecand[i]);
        if (!idx_ok(p, r, p.nr)) continue;
        const unsigned long long k = __ldcg(&p.ekey[r]);
        const int rho = (int)(k >> 32);
        if (idx_ok(p, rho, p.nc) && __ldcg(&p.dkey[rho]) == (unsigned long long)(unsigned)r) {
            __stcg(&p.rmatch[r], -2);
            __stcg(&p.pred[r], (int)(unsigned)(k & 0xffffffffull));
            __stcg(&p.level[rho], -r);
            push_end(r);
        }
        __stcg(&p.ekey[r], DKEY_NONE);
    }
}
__device__ __forceinline__ void step_det_offer(const Params& p, int n) {
    det_offer(p, n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
__device__ __forceinline__ void step_det_take(const Params& p, int n, int32_t* ep_ctr) {
    det_take(p, n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
             [&](int r) { push(p.endpoints, 0, ep_ctr, r); });
}

// ------------------------------------------------------------------ Alternate
// Algorithm 3 over the endpoint list: walk from each endpoint row towards the
// root, rematching every column of the path to the row below it.  The walk
// stops at the root (its old match is -1: reading of the paper's loop bound)
// or when the column was already rematched to a row whose predecessor is
// this column (another walk got there first: the paper's check).
__device__ __forceinline__ void step_alternate(const Params& p, int n_ep, int cap, Counters& cnt) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    unsigned steps_done = 0;
    for (int i = tid; i < n_ep; i += nthr) {
        int r = __ldcg(&p.endpoints[i]);
        int steps = 0;
        while (r != -1) {
            if (++steps > cap) { set_error(p.ctl, -4 /*BM_ERR_ITER_LIMIT*/); break; }
            if (!idx_ok(p, r, p.nr)) break;
            const int c = __ldcg(&p.pred[r]);
            if ((unsigned)c >= (unsigned)p.nc) { set_error(p.ctl, -7 /*BM_ERR_STATE*/); break; }
            const int r2 = ld_volatile(&p.cmatch[c]);
            if (r2 >= 0 && !idx_ok(p, r2, p.nr)) break;
            if (r2 >= 0 && __ldcg(&p.pred[r2]) == c) break;
            st_volatile(&p.cmatch[c], r);
            __stcg(&p.rmatch[r], c);
            ++steps_done;
            r = r2;
        }
    }
    add_to_counter(&p.ctl->alt_steps, steps_done);
}

// Alternate for disjoint search trees (one endpoint per root, Section 3's
// refinement): the walks cannot meet, so a walk needs no meeting check and
// follows the per-column records written by the BFS, one 8-byte load per
// step: column c on the path has (parent column, its old matched row); c is
// rematched to the row below it, and the walk continues from the old row's
// parent.  The root's record is (-1, -1).
__device__ __forceinline__ void step_alternate_disjoint(const Params& p, int n_ep, int cap) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    unsigned steps_done = 0;
    for (int i = tid; i < n_ep; i += nthr) {
        int r = __ldcg(&p.endpoints[i]);
        if (!idx_ok(p, r, p.nr)) continue;
        int c = __ldcg(&p.pred[r]);
        int steps = 0;
        for (;;) {
            if (++steps > cap) { set_error(p.ctl, -4 /*BM_ERR_ITER_LIMIT*/); break; }
            if ((unsigned)c >= (unsigned)p.nc) { set_error(p.ctl, -7 /*BM_ERR_STATE*/); break; }
            const int2 rec = __ldcg(&p.crec[c]);
            __stcg(&p.cmatch[c], r);
            __stcg(&p.rmatch[r], c);
            ++steps_done;
            if (rec.y < 0) break;  // c was the root
            if (!idx_ok(p, rec.y, p.nr)) break;
            r = rec.y;
            c = rec.x;
        }
    }
    add_to_counter(&p.ctl->alt_steps, steps_done);
}

// ------------------------------------------------------------------ FixMatching
// Row half of FixMatching (Section 3): rmatch[r] = -1 wherever
// cmatch[rmatch[r]] != r; a row still marked -2 (its walk stopped at once)
// becomes -1 as well.
__device__ __forceinline__ void step_fix_rows(const Params& p, Counters& cnt) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    unsigned fixes = 0;
    for (int r = tid; r < p.nr; r += nthr) {
        const int m = __ldcg(&p.rmatch[r]);
        if (m == -1) continue;
        if (m < 0 || !idx_ok(p, m, p.nc) || __ldcg(&p.cmatch[m]) != r) {
            __stcg(&p.rmatch[r], -1);
            ++fixes;
        }
    }
    add_to_counter(&p.ctl->fix_repairs, fixes);
}

// Range-checked build: between phases the matching must be consistent --
// every matched row's column points back to it and the other way round.
// A violation records BM_ERR_CHECK.
__device__ __forceinline__ void step_check_matching(const Params& p) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    bool bad = false;
    for (int r = tid; r < p.nr; r += nthr) {
        const int m = __ldcg(&p.rmatch[r]);
        if (m != -1 && (m < 0 || m >= p.nc || __ldcg(&p.cmatch[m]) != r)) bad = true;
    }
    for (int c = tid; c < p.nc; c += nthr) {
        const int m = __ldcg(&p.cmatch[c]);
        if (m != -1 && (m < 0 || m >= p.nr || __ldcg(&p.rmatch[m]) != c)) bad = true;
    }
    if (bad && p.chk) atomicCAS(p.chk, 0, -11 /*BM_ERR_CHECK*/);
}

// Gives back the rows a BFS-only pass claimed (inspection entry point).
__device__ __forceinline__ void step_release_endpoints(const Params& p, int n_ep) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    for (int i = tid; i < n_ep; i += nthr) {
        const int r = __ldcg(&p.endpoints[i]);
        if (idx_ok(p, r, p.nr)) __stcg(&p.rmatch[r], -1);
    }
}

// ------------------------------------------------------------------ one graph, one block
// InitBfsArray over all columns of one graph by one block (4 columns per
// thread in flight): column half of FixMatching, level / root init, unmatched
// columns with rows appended to the queue as roots.  Returns the roots in
// sm.qn; free_total / iso_free get all unmatched columns and those without rows.
// SB: the search keeps its tree marks in the shared-memory bitmaps, so the
// columns' level and root entries are not written.
template <bool WR, bool NC, bool SB = false>
__device__ __forceinline__ void block_full_init(const Params& p, Smem& sm, Counters& cnt, int& free_total,
                                                int& iso_free) {
    const int T = blockDim.x, t = threadIdx.x, nc = p.nc;
    if (t == 0) { sm.qn = 0; sm.qbase = 0; sm.total = 0; sm.tile = 0; }
    __syncthreads();
    int nfree = 0, niso = 0;
    for (int base = 0; base < nc; base += 4 * T) {
        int c[4], r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = base + u * T + t;
            r[u] = c[u] < nc ? __ldcg(&p.cmatch[c[u]]) : -3;
            if (r[u] >= 0 && !idx_ok(p, r[u], p.nr)) r[u] = -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] >= nc) continue;
            if (r[u] >= 0 && __ldcg(&p.rmatch[r[u]]) != c[u]) {
                __stcg(&p.cmatch[c[u]], -1);
                r[u] = -1;
                cnt.fixes++;
            }
            const bool is_free = r[u] < 0;
            if (!SB) {
                __stcg(&p.level[c[u]], is_free ? L0 : L0 - 1);
                if (WR) __stcg(&p.root[c[u]], is_free ? c[u] : -1);
            }
            if (is_free) {
                ++nfree;
                if (ld_csr<NC>(&p.col_ptr[c[u] + 1]) > ld_csr<NC>(&p.col_ptr[c[u]]))
                    p.queue[atomicAdd(&sm.qn, 1)] = make_int2(c[u], c[u]);
                else
                    ++niso;
            }
        }
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        nfree += __shfl_down_sync(FULL, nfree, s);
        niso += __shfl_down_sync(FULL, niso, s);
    }
    if ((t & 31) == 0 && nfree) atomicAdd(&sm.total, nfree);
    if ((t & 31) == 0 && niso) atomicAdd(&sm.tile, niso);
    __syncthreads();
    free_total = sm.total;
    iso_free = sm.tile;
    __syncthreads();
}

// The whole method on one graph by one block (batched and served paths):
// optional cheap matching, then Algorithm 1 with the steps separated by
// __syncthreads; queue tail and endpoint count live in shared memory (sm.qn,
// sm.qbase).  With GPUBFS-WR and one endpoint per root, the search trees are
// disjoint and each holds at most one endpoint, so Alternate's walks never
// meet: every walk reaches its root and FixMatching has nothing to repair.
// That mode therefore skips the FixMatching passes and, instead of
// re-initialising every column each phase, resets the columns the last
// search visited and keeps the roots that are still unmatched (work per phase
// proportional to the search, not to n_cols).  The other modes run the full
// passes.  Returns the graph's status.
// CA: the tile expansion reads rows' matches and columns' levels through L1.
// Only when no other block writes the graph's arrays during the launch and the
// memory is not reused for another graph within it (the batched kernel: the
// block's own writes and atomics keep its SM's L1 coherent, and every launch
// starts with a clean L1); the serving workers recycle pool memory within one
// launch and read through L2.
// SB: one endpoint per root with the graph's tree and served-root marks in
// the shared-memory bitmaps p.vis / p.srv (at most SB_MAX_COLS columns):
// cleared at each search's start, the roots' bits set, and the column levels
// neither tested nor reset.
template <bool WR, bool NC, bool CA = false, bool SB = false>
__device__ int block_match_graph(const Params& p, int greedy, Smem& sm, Counters& cnt, int& card_out,
                                 int& phases_out, long long& levels_out, long long& eps_out,
                                 long long& ins_out) {
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int nr = p.nr, nc = p.nc;
    const bool incremental = WR && p.one_ep;
    // SB with rows that fit the bitmap: until the search starts, p.vis marks the
    // rows that are matched, so the cheap matching tests and claims a row in
    // shared memory instead of loading and CASing its match
    const bool rows_sb = SB && nr <= SB_MAX_COLS;
    if (t == 0) sm.ok = 0;
    // ---- rows whose column does not point back are unmatched (row half of FixMatching)
    if (rows_sb) {  // a warp takes 32 consecutive rows and writes their bitmap word
        const int lane = t & 31;
        for (int r0 = t - lane; r0 < nr; r0 += T) {  // warp-uniform: blockDim is a multiple of 32
            const int r = r0 + lane;
            int m = r < nr ? __ldcg(&p.rmatch[r]) : -1;
            if (m != -1 && (m < 0 || m >= nc || __ldcg(&p.cmatch[m]) != r)) {
                __stcg(&p.rmatch[r], -1);
                m = -1;
            }
            const unsigned w = __ballot_sync(FULL, m != -1);
            if (lane == 0) p.vis[r0 >> 5] = w;
        }
    } else {
        for (int r = t; r < nr; r += T) {
            const int m = __ldcg(&p.rmatch[r]);
            if (m != -1 && (m < 0 || m >= nc || __ldcg(&p.cmatch[m]) != r)) __stcg(&p.rmatch[r], -1);
        }
    }
    __syncthreads();
    // ---- cheap matching (Section 4): unmatched columns claim their first free row.
    // A thread walks the lists of GU columns together, GW rows of each per step,
    // so that GU x GW row loads (and, without rows_sb, then GU x GW match loads)
    // are in flight at once and a thread takes as long as its longest walk / GW
    // (not the sum of its walks).  A column's row range is loaded beside its match.
    // rows_sb: a row's test and claim are a bitmap read and atomicOr in shared
    // memory, and the winner stores both matches (read only after the block barrier).
    if (greedy) {
        constexpr int GW = 8, GU = 2;
        for (int base = 0; base < nc; base += GU * T) {
            int c[GU], pos[GU], e[GU];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                c[u] = base + u * T + t;
                pos[u] = e[u] = 0;
                int m0 = 0;
                if (c[u] < nc) {  // the row range is loaded beside the match, not after it
                    m0 = __ldcg(&p.cmatch[c[u]]);
                    pos[u] = ld_csr<NC>(&p.col_ptr[c[u]]);
                    e[u] = ld_csr<NC>(&p.col_ptr[c[u] + 1]);
                }
                if (m0 != -1) e[u] = pos[u];
            }
            for (;;) {
                int r[GU][GW], m[GU][GW];
#pragma unroll
                for (int u = 0; u < GU; ++u)
#pragma unroll
                    for (int k = 0; k < GW; ++k) r[u][k] = pos[u] + k < e[u] ? ld_csr<NC>(&p.row_idx[pos[u] + k]) : -1;
#pragma unroll
                for (int u = 0; u < GU; ++u)
#pragma unroll
                    for (int k = 0; k < GW; ++k)
                        m[u][k] = r[u][k] < 0 ? 0 : rows_sb ? (sb_test(p.vis, r[u][k]) ? 0 : -1)
                                                            : ld_volatile(&p.rmatch[r[u][k]]);
                bool more = false;
#pragma unroll
                for (int u = 0; u < GU; ++u) {
                    if (pos[u] >= e[u]) continue;
                    bool got = false;
#pragma unroll
                    for (int k = 0; k < GW; ++k) {  // the first free row of the window, in list order
                        if (got || m[u][k] != -1) continue;
                        if (rows_sb ? sb_claim(p.vis, r[u][k]) : atomicCAS(&p.rmatch[r[u][k]], -1, c[u]) == -1) {
                            if (rows_sb) p.rmatch[r[u][k]] = c[u];
                            p.cmatch[c[u]] = r[u][k];
                            got = true;
                        }
                    }
                    pos[u] = got ? e[u] : pos[u] + GW;
                    more |= pos[u] < e[u];
                }
                if (!more) break;
            }
        }
    }
    __syncthreads();
    const int max_phases = (nr < nc ? nr : nc) + 2;
    int phases = 0, card = 0, status = 0;
    long long levels_total = 0, eps_total = 0, ins_total = 0;
    int free_total = 0, iso_free = 0;
    block_full_init<WR, NC, SB>(p, sm, cnt, free_total, iso_free);
    int n_roots = sm.qn;
    for (;;) {
        card = nc - free_total;
        if (n_roots == 0) break;
        if (phases >= max_phases) { status = -4 /*BM_ERR_ITER_LIMIT*/; break; }
        ++phases;
        // ---- BFS levels; sm.qn is the queue tail, sm.qbase the endpoint count
        if (t == 0) { sm.qn = n_roots; sm.qbase = 0; sm.grab[0] = 0; sm.nhub[0] = 0; }
        if (SB) {
            for (int w = t; w < (nc + 31) >> 5; w += T) { p.vis[w] = 0u; p.srv[w] = 0u; }
            __syncthreads();
            for (int i = t; i < n_roots; i += T) {
                const int c = __ldcg(&p.queue[i]).x;
                if (idx_ok(p, c, nc)) atomicOr(&p.vis[c >> 5], 1u << (c & 31));
            }
        }
        __syncthreads();
        int qb = 0, qe = n_roots, lvl = L0, levels = 0, n_ep = 0;
        auto push_col = [&](int2 v) { p.queue[atomicAdd(&sm.qn, 1)] = v; };
        auto push_end = [&](int v) { p.endpoints[atomicAdd(&sm.qbase, 1)] = v; };
        for (;;) {
            const int q = qe - qb;
            const bool wide = q > T && 2 * T <= MAX_BLOCK;  // two queue entries per thread
            const int tw = wide ? 2 * T : T;
            int nh = 0;
            if (SB) {  // by warps; the other counters are zeroed for the next level
                if (t == 0) { sm.grab[(levels + 1) & 1] = 0; sm.nhub[(levels + 1) & 1] = 0; }
                warp_expand_sb<NC, CA>(p, qb, q, &sm.grab[levels & 1], &sm.nhub[levels & 1], sm, cnt, push_col,
                                       push_end);
                __syncthreads();
                nh = min(sm.nhub[levels & 1], HUB_MAX);  // block-uniform: reset only after the barrier below
                if (nh > 0) block_hubs_sb<NC, CA>(p, nh, sm, cnt, push_col, push_end);
            }
            for (int first = 0; first < q && !SB; first += tw) {
                if (wide) tile_load2<WR, NC>(p, p.queue, qb, q, first, sm, cnt);
                else tile_load<WR, NC>(p, p.queue, qb, q, first, T, sm, cnt, nullptr);
                tile_edges<WR, decltype(push_col), decltype(push_end), NC, false, CA>(p, tw, lvl, q <= T, sm, cnt,
                                                                                 push_col, push_end);
                __syncthreads();  // sm.off/beg/col/root are reused by the next tile
            }
            if (!SB || nh > 0) __syncthreads();
            const int tail = sm.qn;
            const int eps = sm.qbase;
            // SB: no barrier precedes the next level's appends (the warps start at
            // once), so every thread reads the tail, the endpoint count and the hub
            // count before any warp goes on
            if (SB) __syncthreads();
            ++levels;
            ins_total += tail - qe;
            if (tail == qe) { n_ep = eps; break; }  // no vertex inserted
            if (p.mode == 1 && eps > 0) { n_ep = eps; break; }  // APsB
            if (levels > nc + 2) { status = -4; n_ep = eps; break; }
            qb = qe;
            qe = tail;
            ++lvl;
        }
        const int tail = sm.qn;
        levels_total += levels;
        eps_total += n_ep;
        if (status) break;
        if (n_ep == 0) break;  // no augmenting path: maximum (Berge)
        // ---- Alternate (Algorithm 3)
        for (int i = t; i < n_ep; i += T) {
            int r = __ldcg(&p.endpoints[i]);
            int steps = 0;
            while (r != -1) {
                if (++steps > tail + 2) { atomicCAS(&sm.ok, 0, -4); break; }
                if (!idx_ok(p, r, nr)) { atomicCAS(&sm.ok, 0, -11); break; }
                const int c = __ldcg(&p.pred[r]);
                if ((unsigned)c >= (unsigned)nc) { atomicCAS(&sm.ok, 0, -7); break; }
                const int r2 = ld_volatile(&p.cmatch[c]);
                if (r2 >= 0 && !idx_ok(p, r2, nr)) { atomicCAS(&sm.ok, 0, -11); break; }
                if (r2 >= 0 && __ldcg(&p.pred[r2]) == c) break;
                st_volatile(&p.cmatch[c], r);
                __stcg(&p.rmatch[r], c);
                cnt.alt++;
                r = r2;
            }
        }
        __syncthreads();
        if (sm.ok != 0) { status = sm.ok; break; }
        if (incremental) {
            // columns inserted by this search go back to "unvisited" (SB: the bitmaps are
            // cleared when the next search starts) ...
            for (int i = n_roots + t; i < tail && !SB; i += T) {
                const int c = __ldcg(&p.queue[i]).x;
                if (!idx_ok(p, c, nc)) continue;
                __stcg(&p.level[c], L0 - 1);
                if (WR) __stcg(&p.root[c], -1);
            }
            // ... and the roots that are still unmatched stay roots (compacted in place:
            // entry i moves to a position <= i, after every entry up to i has been read)
            int kept = 0;
            for (int base = 0; base < n_roots; base += T) {
                const int i = base + t;
                int c = -1, keep = 0;
                if (i < n_roots) {
                    c = __ldcg(&p.queue[i]).x;
                    if (!idx_ok(p, c, nc)) c = 0;  // checked build only: recorded, and column 0 is harmless here
                    keep = __ldcg(&p.cmatch[c]) < 0;
                    if (!keep && !SB) {
                        __stcg(&p.level[c], L0 - 1);
                        if (WR) __stcg(&p.root[c], -1);
                    }
                }
                const int pos = block_exclusive_scan(keep, sm);
                const int chunk = sm.total;
                if (keep) p.queue[kept + pos] = make_int2(c, c);
                kept += chunk;
                __syncthreads();
            }
            n_roots = kept;
            free_total = iso_free + kept;
        } else {
            // ---- row half of FixMatching, then InitBfsArray over every column
            for (int r = t; r < nr; r += T) {
                const int m = __ldcg(&p.rmatch[r]);
                if (m == -1) continue;
                if (m < 0 || __ldcg(&p.cmatch[m]) != r) {
                    __stcg(&p.rmatch[r], -1);
                    cnt.fixes++;
                }
            }
            __syncthreads();
            block_full_init<WR, NC, SB>(p, sm, cnt, free_total, iso_free);
            n_roots = sm.qn;
        }
    }
    card_out = card;
    phases_out = phases + (n_roots == 0 ? 1 : 0);  // no root left: Algorithm 1's last search finds nothing
    levels_out = levels_total;
    eps_out = eps_total;
    ins_out = ins_total;
    __syncthreads();
    return status;
}

// ------------------------------------------------------------------ one graph, one block, deterministic
// The cheap matching of the deterministic option, by one block: rounds in
// which every unmatched column proposes to the first unmatched row of its
// list and every proposed row takes the smallest proposer (atomicMin in
// ekey[r]); until a round without proposals.  Columns of more than 32 rows
// look for their row a warp at a time (32 rows per step, a ballot of the free
// ones), from a list in the queue buffer; the others a thread each.
// Scratch: level (position in the column's list), root (the row proposed to,
// -1 none); ekey must be all ones before and is again after.
template <bool NC>
__device__ __forceinline__ void block_greedy_rounds(const Params& p, Smem& sm) {
    const int T = blockDim.x, t = threadIdx.x, nc = p.nc;
    const int lane = t & 31, warp = t >> 5, nwarps = (T + 31) >> 5;
    int32_t* longs = (int32_t*)p.queue;
    if (t == 0) sm.tile = 0;
    __syncthreads();
    for (int c = t; c < nc; c += T) {
        const int b = ld_csr<NC>(&p.col_ptr[c]);
        __stcg(&p.level[c], b);
        if (ld_csr<NC>(&p.col_ptr[c + 1]) - b > 32) longs[atomicAdd(&sm.tile, 1)] = c;
    }
    __syncthreads();
    const int nlong = sm.tile;
    for (int round = 0; round <= nc; ++round) {
        if (t == 0) sm.ok = 0;
        __syncthreads();
        bool any = false;
        for (int c = t; c < nc; c += T) {  // short lists: a thread each
            const int end = ld_csr<NC>(&p.col_ptr[c + 1]);
            if (end - ld_csr<NC>(&p.col_ptr[c]) > 32) continue;
            int want = -1;
            if (__ldcg(&p.cmatch[c]) == -1) {
                int pos = __ldcg(&p.level[c]);
                while (pos < end) {  // 4 rows per step, their matches in flight together
                    int r[4], m[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) r[u] = pos + u < end ? ld_csr<NC>(&p.row_idx[pos + u]) : -1;
#pragma unroll
                    for (int u = 0; u < 4; ++u) m[u] = (r[u] >= 0 && idx_ok(p, r[u], p.nr)) ? __ldcg(&p.rmatch[r[u]]) : 0;
                    int k = 0;
                    while (k < 4 && r[k] >= 0 && m[k] != -1) ++k;
                    if (k < 4 && r[k] >= 0) { pos += k; want = r[k]; break; }
                    pos += 4;
                }
                if (pos > end) pos = end;
                __stcg(&p.level[c], pos);
                if (want >= 0) {
                    atomicMin(&p.ekey[want], (unsigned long long)(unsigned)c);
                    any = true;
                }
            }
            __stcg(&p.root[c], want);
        }
        for (int k = warp; k < nlong; k += nwarps) {  // long lists: a warp each (warp-uniform)
            const int c = __ldcg(&longs[k]);
            if (!idx_ok(p, c, nc)) continue;
            int want = -1;
            if (__ldcg(&p.cmatch[c]) == -1) {
                const int end = ld_csr<NC>(&p.col_ptr[c + 1]);
                int pos = __ldcg(&p.level[c]);
                while (pos < end) {
                    const int r = pos + lane < end ? ld_csr<NC>(&p.row_idx[pos + lane]) : -1;
                    const int m = (r >= 0 && idx_ok(p, r, p.nr)) ? __ldcg(&p.rmatch[r]) : 0;
                    const unsigned free_rows = __ballot_sync(FULL, r >= 0 && m == -1);
                    if (free_rows) {
                        const int k0 = __ffs(free_rows) - 1;
                        pos += k0;
                        want = __shfl_sync(FULL, r, k0);
                        break;
                    }
                    pos += 32;
                }
                if (pos > end) pos = end;
                if (lane == 0) {
                    __stcg(&p.level[c], pos);
                    if (want >= 0) atomicMin(&p.ekey[want], (unsigned long long)(unsigned)c);
                }
                if (want >= 0) any = true;
            }
            if (lane == 0) __stcg(&p.root[c], want);
        }
        if (any) sm.ok = 1;
        __syncthreads();
        const bool more = sm.ok != 0;
        for (int c = t; c < nc; c += T) {
            const int r = __ldcg(&p.root[c]);
            if (r >= 0 && __ldcg(&p.ekey[r]) == (unsigned long long)(unsigned)c) {
                __stcg(&p.rmatch[r], c);
                __stcg(&p.cmatch[c], r);
            }
        }
        __syncthreads();
        for (int c = t; c < nc; c += T) {
            const int r = __ldcg(&p.root[c]);
            if (r >= 0) __stcg(&p.ekey[r], DKEY_NONE);
        }
        __syncthreads();
        if (!more) break;
    }
}

// The whole method on one graph by one block with the deterministic option's
// rules (GPUBFS-WR, one endpoint per root; p.dkey, p.ekey, p.ecand hold the
// graph's keys and offer list): the cheap matching in rounds if `greedy`,
// then Algorithm 1 one level at a time, each level followed -- when it
// produced offers -- by the two passes that hand rows to roots.  The search
// trees are disjoint, so Alternate's walks never meet.  Same outputs as
// block_match_graph; the result depends on the graph and the start only.
// SB: p.vis (shared memory, at most SB_MAX_COLS columns) marks the columns of
// the levels searched so far, so that edges into them skip the claim word.
template <bool NC, bool SB = false>
__device__ int block_match_graph_det(const Params& p, int greedy, Smem& sm, Counters& cnt, int& card_out,
                                     int& phases_out, long long& levels_out, long long& eps_out,
                                     long long& ins_out) {
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int nr = p.nr, nc = p.nc;
    if (t == 0) sm.ok = 0;
    // ---- rows whose column does not point back are unmatched; every key "none"
    for (int r = t; r < nr; r += T) {
        const int m = __ldcg(&p.rmatch[r]);
        if (m != -1 && (m < 0 || m >= nc || __ldcg(&p.cmatch[m]) != r)) __stcg(&p.rmatch[r], -1);
        __stcg(&p.ekey[r], DKEY_NONE);
    }
    for (int c = t; c < nc; c += T) __stcg(&p.dkey[c], DKEY_NONE);
    __syncthreads();
    if (greedy) block_greedy_rounds<NC>(p, sm);
    if (t == 0) sm.ok = 0;  // the rounds used it as their flag; from here it holds Alternate's errors
    const int max_phases = (nr < nc ? nr : nc) + 2;
    int phases = 0, card = 0, status = 0;
    long long levels_total = 0, eps_total = 0, ins_total = 0;
    int free_total = 0, iso_free = 0;
    block_full_init<true, NC>(p, sm, cnt, free_total, iso_free);
    int n_roots = sm.qn;
    for (;;) {
        card = nc - free_total;
        if (n_roots == 0) break;
        if (phases >= max_phases) { status = -4 /*BM_ERR_ITER_LIMIT*/; break; }
        ++phases;
        // sm.qn: queue tail; sm.qbase: endpoints; sm.npush: rows listed in ecand this level
        if (t == 0) { sm.qn = n_roots; sm.qbase = 0; sm.npush = 0; sm.has_ep = 0; sm.grab[0] = 0; sm.nhub[0] = 0; }
        __syncthreads();
        int qb = 0, qe = n_roots, lvl = L0, levels = 0, n_ep = 0;
        auto push_col = [&](int2 v) { p.queue[atomicAdd(&sm.qn, 1)] = v; };
        auto push_off = [&](int r) { p.ecand[atomicAdd(&sm.npush, 1)] = r; };
        auto push_end = [&](int r) { p.endpoints[atomicAdd(&sm.qbase, 1)] = r; };
        // a queue entry of a level after L0 carries no root yet: it is completed from
        // the column's tree-entry word (as tile_load_det), then the GPUBFS-WR root test
        auto entry_det = [&](int2 e, int& c, int& rt, int& beg, int& deg) {
            c = e.x;
            if (!idx_ok(p, c, nc)) {  // checked build only
                c = -1;
                return;
            }
            beg = ld_csr<NC>(&p.col_ptr[c]);
            deg = ld_csr<NC>(&p.col_ptr[c + 1]) - beg;
            if (lvl == L0) {
                rt = e.y;  // a root: (c, c)
            } else {
                const unsigned long long k = __ldcg(&p.dkey[c]);
                const int par = (int)(unsigned)(k & 0xffffffffull);
                const int row = __ldcg(&p.cmatch[c]);
                if (!idx_ok(p, par, nc) || !idx_ok(p, row, nr)) {
                    c = -1;
                    return;
                }
                rt = __ldcg(&p.root[par]);
                __stcg(&p.root[c], rt);
                __stcg(&p.level[c], lvl);
                __stcg(&p.pred[row], par);
                if (p.crec) __stcg(&p.crec[c], make_int2(par, row));
            }
            if (!idx_ok(p, rt, nc) || __ldcg(&p.level[rt]) < L0 - 1) c = -1;  // Algorithm 4: root served
        };
        // the edges as tile_edges_det: smallest (level, parent) claims a column, smallest
        // (root, column) an unmatched row's offer
        auto round_det = [&](const int (&own)[ILP], const int (&r)[ILP], const int* s_col, const int* s_root) {
            const unsigned long long next_lv = (unsigned long long)(unsigned)(lvl + 1) << 32;
            int cm[ILP];
            unsigned long long key[ILP];
#pragma unroll
            for (int u = 0; u < ILP; ++u) cm[u] = own[u] >= 0 ? __ldcg(&p.rmatch[r[u]]) : -3;
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                if (cm[u] >= 0 && !idx_ok(p, cm[u], nc)) cm[u] = -3;  // checked build only
#pragma unroll
            for (int u = 0; u < ILP; ++u)
                key[u] = (cm[u] < 0 || (SB && sb_test(p.vis, cm[u]))) ? 0ull : __ldcg(&p.dkey[cm[u]]);
#pragma unroll
            for (int u = 0; u < ILP; ++u) {
                if (own[u] < 0) continue;
                const int col = s_col[own[u]];
                cnt.edges++;
                if (cm[u] >= 0) {
                    cnt.em++;
                    // keys only decrease: a stale key that is not above ours is final
                    const unsigned long long want = next_lv | (unsigned)col;
                    if (key[u] > want && atomicMin(&p.dkey[cm[u]], want) == DKEY_NONE) push_col(make_int2(cm[u], -1));
                } else if (cm[u] == -1) {
                    const unsigned long long want = ((unsigned long long)(unsigned)s_root[own[u]] << 32) | (unsigned)col;
                    if (atomicMin(&p.ekey[r[u]], want) == DKEY_NONE) push_off(r[u]);
                }
            }
        };
        auto alive_det = [](int) { return true; };  // a root is served only between levels (det_take)
        if (SB) {  // a new search: no column in a tree yet
            for (int w = t; w < (nc + 31) >> 5; w += T) p.vis[w] = 0u;
            __syncthreads();
        }
        for (;;) {
            const int q = qe - qb;
            if (SB) {  // the level's own columns join the marked ones before its edges are read
                for (int i = t; i < q; i += T) {
                    const int c = __ldcg(&p.queue[qb + i]).x;
                    if (idx_ok(p, c, nc)) atomicOr(&p.vis[c >> 5], 1u << (c & 31));
                }
                __syncthreads();
            }
            // by warps; the other counters are zeroed for the next level
            if (t == 0) { sm.grab[(levels + 1) & 1] = 0; sm.nhub[(levels + 1) & 1] = 0; }
            warp_expand<NC>(p, qb, q, &sm.grab[levels & 1], &sm.nhub[levels & 1], sm, cnt, entry_det, round_det);
            __syncthreads();
            const int nh = min(sm.nhub[levels & 1], HUB_MAX);  // reset only after the barrier that ends the level
            if (nh > 0) {
                block_hubs<NC>(p, nh, sm, alive_det, round_det);
                __syncthreads();
            }
            const int n_off = sm.npush;
            const bool found = n_off > 0;
            if (found) {
                det_offer(p, n_off, t, T);
                __syncthreads();
                det_take(p, n_off, t, T, push_end);
                __syncthreads();
                if (t == 0) { sm.npush = 0; sm.has_ep = 0; }
            }
            const int tail = sm.qn;
            const int eps = sm.qbase;
            __syncthreads();
            ++levels;
            ins_total += tail - qe;
            if (tail == qe) { n_ep = eps; break; }          // no vertex inserted
            if (p.mode == 1 && found) { n_ep = eps; break; }  // APsB
            if (levels > nc + 2) { status = -4; n_ep = eps; break; }
            qb = qe;
            qe = tail;
            ++lvl;
        }
        const int tail = sm.qn;
        levels_total += levels;
        eps_total += n_ep;
        if (status) break;
        if (n_ep == 0) break;  // no augmenting path: maximum (Berge)
        // ---- Alternate (Algorithm 3): disjoint paths, each walked to its root
        for (int i = t; i < n_ep; i += T) {
            int r = __ldcg(&p.endpoints[i]);
            int steps = 0;
            while (r != -1) {
                if (++steps > tail + 2) { atomicCAS(&sm.ok, 0, -4); break; }
                if (!idx_ok(p, r, nr)) { atomicCAS(&sm.ok, 0, -11); break; }
                const int c = __ldcg(&p.pred[r]);
                if ((unsigned)c >= (unsigned)nc) { atomicCAS(&sm.ok, 0, -7); break; }
                const int r2 = __ldcg(&p.cmatch[c]);
                __stcg(&p.cmatch[c], r);
                __stcg(&p.rmatch[r], c);
                cnt.alt++;
                r = r2;
            }
        }
        __syncthreads();
        if (sm.ok != 0) { status = sm.ok; break; }
        // ---- columns inserted by this search go back to "unvisited" ...
        for (int i = n_roots + t; i < tail; i += T) {
            const int c = __ldcg(&p.queue[i]).x;
            if (!idx_ok(p, c, nc)) continue;
            __stcg(&p.level[c], L0 - 1);
            __stcg(&p.root[c], -1);
            __stcg(&p.dkey[c], DKEY_NONE);
        }
        // ... and the roots that are still unmatched stay roots (compacted in place)
        int kept = 0;
        for (int base = 0; base < n_roots; base += T) {
            const int i = base + t;
            int c = -1, keep = 0;
            if (i < n_roots) {
                c = __ldcg(&p.queue[i]).x;
                if (!idx_ok(p, c, nc)) c = 0;  // checked build only: recorded, and column 0 is harmless here
                keep = __ldcg(&p.cmatch[c]) < 0;
                __stcg(&p.dkey[c], DKEY_NONE);
                if (!keep) {
                    __stcg(&p.level[c], L0 - 1);
                    __stcg(&p.root[c], -1);
                }
            }
            const int pos = block_exclusive_scan(keep, sm);
            const int chunk = sm.total;
            if (keep) p.queue[kept + pos] = make_int2(c, c);
            kept += chunk;
            __syncthreads();
        }
        n_roots = kept;
        free_total = iso_free + kept;
    }
    card_out = card;
    phases_out = phases + (n_roots == 0 ? 1 : 0);
    levels_out = levels_total;
    eps_out = eps_total;
    ins_out = ins_total;
    __syncthreads();
    return status;
}

// Checks one graph's CSR with one block: col_ptr from 0, monotone, up to nnz
// (so every later row_idx read is in range), rows in [0, nr).  Returns
// whether it is valid (same answer in every thread).
template <bool NC>
__device__ bool block_check_csr(int nr, int nc, long long nnz, const int32_t* cp, const int32_t* ri, Smem& sm) {
    if (threadIdx.x == 0) sm.ok = (nr < 0 || nc < 0 || ld_csr<NC>(&cp[0]) != 0 ||
                                   (long long)ld_csr<NC>(&cp[nc]) != nnz) ? 1 : 0;
    __syncthreads();
    bool bad = false;
    if (sm.ok == 0) {
        for (int c = threadIdx.x; c < nc; c += blockDim.x)
            if (ld_csr<NC>(&cp[c + 1]) < ld_csr<NC>(&cp[c])) bad = true;
    }
    if (bad) atomicOr(&sm.ok, 1);
    __syncthreads();
    if (sm.ok == 0) {
        for (long long e = threadIdx.x; e < nnz; e += blockDim.x) {
            const int r = ld_csr<NC>(&ri[e]);
            if (r < 0 || r >= nr) bad = true;
        }
    }
    if (bad) atomicOr(&sm.ok, 1);
    __syncthreads();
    const bool ok = sm.ok == 0;
    __syncthreads();
    return ok;
}

__device__ __forceinline__ void flush_counters(const Params& p, Counters& cnt) {
    // one atomic per warp
    unsigned long long a = cnt.cols, b = cnt.edges, f = cnt.fixes, m = cnt.em, t = cnt.alt;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        a += __shfl_down_sync(FULL, a, s);
        b += __shfl_down_sync(FULL, b, s);
        f += __shfl_down_sync(FULL, f, s);
        m += __shfl_down_sync(FULL, m, s);
        t += __shfl_down_sync(FULL, t, s);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd((unsigned long long*)&p.ctl->cols_expanded, (unsigned long long)a);
        if (b) atomicAdd((unsigned long long*)&p.ctl->edges_scanned, (unsigned long long)b);
        if (f) atomicAdd((unsigned long long*)&p.ctl->fix_repairs, (unsigned long long)f);
        if (m) atomicAdd((unsigned long long*)&p.ctl->edges_matched, (unsigned long long)m);
        if (t) atomicAdd((unsigned long long*)&p.ctl->alt_steps, (unsigned long long)t);
    }
    cnt = Counters{0, 0, 0, 0, 0};
}

}  // namespace bmd
