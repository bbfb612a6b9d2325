// Device-side building blocks of the matching path (sm_103a).
//
// One phase of Algorithm 1 of arXiv 1303.1379 (Section 3) is
//   InitBfsArray -> BFS levels (Algorithm 2 GPUBFS / Algorithm 4 GPUBFS-WR)
//   -> Alternate (Algorithm 3) -> FixMatching.
// This header holds those steps as device functions over "all threads of the
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
//    the single winner writes pred/root and appends the column (warp-
//    aggregated atomics).  The paper's atomic-free writes let several threads
//    insert the same column; a queue needs exactly one.
//  * Free rows are claimed with a CAS -1 -> -2 on rmatch (the paper's plain
//    store of -2), so every endpoint has exactly one predecessor and is
//    appended once to an endpoint list; Alternate walks that list instead of
//    scanning all rows for -2.
//  * A warp expands 32 queue entries at a time: columns with more than 32
//    rows are scanned by the whole warp, one after another; the rest are
//    expanded by a warp-wide prefix sum over their degrees, so every lane
//    handles one edge per iteration whatever the degree mix.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>

namespace bmd {

namespace cg = cooperative_groups;

constexpr int L0 = 2;  // BFS start level (Section 3 chooses L0 = 2)
constexpr unsigned FULL = 0xffffffffu;

// Control block in device memory, cleared before every launch.  Per-step
// counters rotate over three slots: step s appends to slot s % 3 and clears
// slot (s + 1) % 3, which nobody reads during step s (it was last read right
// after the barrier that ended step s - 2).
struct alignas(128) Ctl {
    unsigned long long bar;  // grid barrier arrivals (monotone)
    int32_t pad_bar[30];
    int32_t qcnt[3];         // columns appended during a step
    int32_t ecnt[3];         // endpoints appended during a step
    int32_t err;             // first error code (0 = none)
    int32_t status;          // final status of the launch
    int32_t card;            // |M| at the end
    int32_t initial_card;
    int32_t phases;
    int32_t n_endpoints_last;  // endpoints of the last BFS (inspection)
    int32_t pad1[18];
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
    int32_t* queue;      // columns of the current phase, level by level
    int32_t* endpoints;  // rows claimed as path ends in the current phase
    Ctl* ctl;
    int32_t mode;        // 0 APFB, 1 APsB
    int32_t one_ep;      // GPUBFS-WR: one endpoint per root (-(row) in the root slot)
    int32_t max_phases;  // stop after this many phases (>= 1)
    int32_t phase_limit_is_error;
    int32_t bfs_only;    // run one BFS, no Alternate, leave the matching as installed
    int32_t pad;
    long long wait_ns;   // limit of one barrier wait
    long long total_ns;  // limit of the whole launch
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

// Appends v at base + (running count of `slot`) with one atomic per group of
// converged lanes.
__device__ __forceinline__ void push(int32_t* buf, int base, int32_t* slot, int v) {
    cg::coalesced_group g = cg::coalesced_threads();
    int pos = 0;
    if (g.thread_rank() == 0) pos = atomicAdd(slot, (int)g.size());
    pos = g.shfl(pos, 0) + (int)g.thread_rank();
    buf[base + pos] = v;
}

// ------------------------------------------------------------------ grid barrier
// All blocks of a cooperative launch.  Returns false (in every thread of the
// block) when the wait ran out of time, the launch deadline passed or any
// block recorded an error; the caller then leaves the kernel.
__device__ __noinline__ bool grid_sync(Ctl* ctl, unsigned long long& target, long long wait_ns,
                                       unsigned long long deadline) {
    __shared__ int s_ok;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(&ctl->bar, 1ull);
        unsigned long long t_end = globaltimer() + (unsigned long long)wait_ns;
        if (t_end > deadline) t_end = deadline;
        unsigned spins = 0;
        while (ld_acquire_u64(&ctl->bar) < target) {
            if ((++spins & 31u) == 0) {
                if (ld_volatile(&ctl->err) != 0) { ok = 0; break; }
                if (globaltimer() > t_end) { set_error(ctl, -5 /*BM_ERR_TIMEOUT*/); ok = 0; break; }
            }
        }
        if (ok && ld_volatile(&ctl->err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct Counters {
    long long cols, edges, fixes, em, alt;
};

// ------------------------------------------------------------------ InitBfsArray
// Algorithm 1 InitBfsArray (+ GPUBFS-WR root init, Section 3): level L0 for
// unmatched columns, L0 - 1 for matched ones; root[c] = c for unmatched ones
// (-1 otherwise: 0 is a valid column id).  Unmatched columns form the first
// queue segment.  Before that, the column half of FixMatching: a column whose
// row does not point back is unmatched (the row half runs after Alternate).
template <bool WR>
__device__ __forceinline__ void step_init(const Params& p, int slot, Counters& cnt) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const int nc = p.nc;
    for (int base = tid - (tid & 31); base < nc; base += nthr) {  // warp-uniform trip count
        int c = base + (threadIdx.x & 31);
        bool is_free = false;
        if (c < nc) {
            int r = __ldcg(&p.cmatch[c]);
            if (r >= 0 && __ldcg(&p.rmatch[r]) != c) {
                __stcg(&p.cmatch[c], -1);
                r = -1;
                cnt.fixes++;
            }
            is_free = (r < 0);
            __stcg(&p.level[c], is_free ? L0 : L0 - 1);
            if (WR) __stcg(&p.root[c], is_free ? c : -1);
        }
        if (is_free) push(p.queue, 0, &p.ctl->qcnt[slot], c);
    }
}

// ------------------------------------------------------------------ BFS level
// Visits edge (row r, column c) of a column c at level lvl whose search tree
// has root `myroot` (GPUBFS-WR).  Algorithm 2 / 4, loop body.
template <bool WR>
__device__ __forceinline__ void visit(const Params& p, int r, int c, int myroot, int lvl,
                                      int qbase, int qslot, int ebase, int eslot, Counters& cnt) {
    int cm = __ldcg(&p.rmatch[r]);
    if (cm >= 0) {
        cnt.em++;
        // matched row: its column joins the next level unless already reached
        if (__ldcg(&p.level[cm]) == L0 - 1 && atomicCAS(&p.level[cm], L0 - 1, lvl + 1) == L0 - 1) {
            __stcg(&p.pred[r], c);
            if (WR) __stcg(&p.root[cm], myroot);
            push(p.queue, qbase, &p.ctl->qcnt[qslot], cm);
        }
    } else if (cm == -1) {
        // unmatched row: an augmenting path ends here
        if (WR && p.one_ep) {
            if (__ldcg(&p.level[myroot]) == L0 && atomicCAS(&p.rmatch[r], -1, -2) == -1) {
                if (atomicCAS(&p.level[myroot], L0, -r) == L0) {
                    __stcg(&p.pred[r], c);
                    push(p.endpoints, ebase, &p.ctl->ecnt[eslot], r);
                } else {
                    atomicExch(&p.rmatch[r], -1);  // root served meanwhile: give the row back
                }
            }
        } else if (atomicCAS(&p.rmatch[r], -1, -2) == -1) {
            if (WR) __stcg(&p.level[myroot], L0 - 2);
            __stcg(&p.pred[r], c);
            push(p.endpoints, ebase, &p.ctl->ecnt[eslot], r);
        }
    }
}

// Expands the queue segment [qb, qe) whose columns are at level lvl.  New
// columns are appended at qe + (slot count), endpoints at ebase + (slot count).
template <bool WR>
__device__ __forceinline__ void step_expand(const Params& p, int qb, int qe, int lvl, int slot,
                                            int ebase, Counters& cnt) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int q = qe - qb;
    for (int base = gwarp * 32; base < q; base += nwarps * 32) {  // warp-uniform
        const int i = base + lane;
        int c = -1, beg = 0, deg = 0, myroot = -1;
        if (i < q) {
            c = __ldcg(&p.queue[qb + i]);
            if (WR) {
                myroot = __ldcg(&p.root[c]);
                if (__ldcg(&p.level[myroot]) < L0 - 1) c = -1;  // Algorithm 4: root already served
            }
            if (c >= 0) {
                beg = __ldg(&p.col_ptr[c]);
                deg = __ldg(&p.col_ptr[c + 1]) - beg;
                cnt.cols++;
            }
        }
        // columns with more than 32 rows: the whole warp scans one at a time
        unsigned big = __ballot_sync(FULL, deg > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int bc = __shfl_sync(FULL, c, src);
            const int bb = __shfl_sync(FULL, beg, src);
            const int bd = __shfl_sync(FULL, deg, src);
            const int br = __shfl_sync(FULL, myroot, src);
            int j0 = 0;
            for (; j0 < bd; j0 += 32) {
                if (WR && j0 != 0 && (j0 & 255) == 0) {  // re-check the root every 256 rows
                    if (__ldcg(&p.level[br]) < L0 - 1) break;
                }
                const int j = j0 + lane;
                if (j < bd) visit<WR>(p, __ldg(&p.row_idx[bb + j]), bc, br, lvl, qe, slot, ebase, slot, cnt);
            }
            if (lane == 0) cnt.edges += (j0 < bd ? j0 : bd);
        }
        if (deg > 32) deg = 0;
        // the rest: warp-wide prefix sum of degrees, one edge per lane per pass
        int incl = deg;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            int v = __shfl_up_sync(FULL, incl, s);
            if (lane >= s) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int off = incl - deg;
        if (lane == 0) cnt.edges += total;
        for (int k = 0; k < total; k += 32) {
            const int e = k + lane;
            int owner = 0;  // last lane whose range starts at or before e
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                int o = __shfl_sync(FULL, off, owner + s);
                if (o <= e) owner += s;
            }
            const int oc = __shfl_sync(FULL, c, owner);
            const int ob = __shfl_sync(FULL, beg, owner);
            const int oo = __shfl_sync(FULL, off, owner);
            const int orr = __shfl_sync(FULL, myroot, owner);
            if (e < total) visit<WR>(p, __ldg(&p.row_idx[ob + (e - oo)]), oc, orr, lvl, qe, slot, ebase, slot, cnt);
        }
    }
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
    for (int i = tid; i < n_ep; i += nthr) {
        int r = __ldcg(&p.endpoints[i]);
        int steps = 0;
        while (r != -1) {
            if (++steps > cap) { set_error(p.ctl, -4 /*BM_ERR_ITER_LIMIT*/); break; }
            const int c = __ldcg(&p.pred[r]);
            if ((unsigned)c >= (unsigned)p.nc) { set_error(p.ctl, -7 /*BM_ERR_STATE*/); break; }
            const int r2 = ld_volatile(&p.cmatch[c]);
            if (r2 >= 0 && __ldcg(&p.pred[r2]) == c) break;
            st_volatile(&p.cmatch[c], r);
            __stcg(&p.rmatch[r], c);
            cnt.alt++;
            r = r2;
        }
    }
}

// ------------------------------------------------------------------ FixMatching
// Row half of FixMatching (Section 3): rmatch[r] = -1 wherever
// cmatch[rmatch[r]] != r; a row still marked -2 (its walk stopped at once)
// becomes -1 as well.
__device__ __forceinline__ void step_fix_rows(const Params& p, Counters& cnt) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    for (int r = tid; r < p.nr; r += nthr) {
        const int m = __ldcg(&p.rmatch[r]);
        if (m == -1) continue;
        if (m < 0 || __ldcg(&p.cmatch[m]) != r) {
            __stcg(&p.rmatch[r], -1);
            cnt.fixes++;
        }
    }
}

// Gives back the rows a BFS-only pass claimed (inspection entry point).
__device__ __forceinline__ void step_release_endpoints(const Params& p, int n_ep) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    for (int i = tid; i < n_ep; i += nthr) __stcg(&p.rmatch[__ldcg(&p.endpoints[i])], -1);
}

__device__ __forceinline__ void flush_counters(const Params& p, Counters& cnt) {
    // one atomic per warp
    long long a = cnt.cols, b = cnt.edges, f = cnt.fixes, m = cnt.em, t = cnt.alt;
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
