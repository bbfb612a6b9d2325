// bmatch: C-ABI of the GPU maximum cardinality bipartite matching path
// (arXiv 1303.1379, Section 3, Algorithms 1-4), written for GB300 (sm_103a).
//
// Two drivers run the same device steps (bm_device.cuh):
//  * persistent (default): ONE cooperative launch per bm_match runs every
//    phase and every BFS level of Algorithm 1 on the device, separated by a
//    software grid barrier whose waits are bounded by %globaltimer.  The host
//    is not involved between levels (the paper reads the flags back after
//    every level).
//  * host: the paper's structure -- one launch per step, the host reads the
//    level counters after each BFS level.  Kept for the variant comparison.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "bm_device.cuh"
#include "bm_internal.h"
#include "bmatch.h"

using bmd::Counters;
using bmd::Ctl;
using bmd::L0;
using bmd::Params;
using bmd::Smem;

namespace {

constexpr int kVersion = 1 * 10000 + 0 * 100 + 0;
constexpr int kDefaultBlock = 512;
constexpr int kProfileCap = 4096;

// ------------------------------------------------------------------ kernels

// Statistics of a persistent launch, kept by its leader thread in shared
// memory (not in every thread's registers: the BFS loop needs them for
// nothing else).
struct LeaderStats {
    unsigned long long t_start;
    long long levels_total, levels_max, eps_total, ins_total, roots_total;
    int levels, first_ep, last_ep;
};

// One launch per match: Algorithm 1 with both loops on the device.  RV: small
// BFS levels claim columns through the row stamps p.rvis (a context's
// launches); without it every level claims through the column levels (the
// allocation-free entry point).  DET: the deterministic option (GPUBFS-WR
// with one endpoint per root; p.dkey, p.ekey and p.ecand set): each level
// is followed, when it produced offers, by the two passes that hand rows to
// roots.
template <bool WR, bool RV, bool DET = false>
__global__ void __launch_bounds__(1024, 1) k_match(Params p) {
    using namespace bmd;
    Ctl* ctl = p.ctl;
    __shared__ Smem sm;
    __shared__ LeaderStats ls;  // written by the leader thread only
    if (threadIdx.x == 0) { sm.qn = 0; sm.npush = 0; sm.has_ep = 0; }
    int bid = 0;  // grid barriers passed
    const unsigned long long deadline = globaltimer() + (unsigned long long)p.total_ns;
    const bool leader = (blockIdx.x == 0 && threadIdx.x == 0);
    if (leader) ls = LeaderStats{globaltimer(), 0, 0, 0, 0, 0, 0, 0, 0};
    // one-endpoint GPUBFS-WR: no FixMatching passes, roots carried to the next phase
    const bool incr = WR && p.one_ep && p.queue2 != nullptr && !p.bfs_only;
    int2* qcur = p.queue;
    int2* qnext = p.queue2;
    Counters cnt{0, 0, 0, 0, 0};
    int step = 0;
    int phases = 0;
    int card = 0;
    int status = 0;
    int n_roots = 0;
    int iso_free = 0;
    int no_roots = 0;  // the loop ended because no column was left to search from
    if (ld_volatile(&ctl->err) != 0) goto out;  // input validation failed before launch
    {
        // ---- InitBfsArray (+ column half of FixMatching)
        const int s = step++;
        if (leader) {
            ctl->qcnt[(s + 1) % 3] = 0;
            ctl->ecnt[(s + 1) % 3] = 0;
            ctl->icnt[(s + 1) % 3] = 0;
            ctl->tcnt[(s + 1) % 3] = 0;
            if (DET) ctl->dcnt[(s + 1) % 3] = 0;
            ctl->ep_phase = 0;
        }
        step_init<WR>(p, qcur, s % 3, cnt, sm);
        if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, &ctl->ecnt[s % 3], &ctl->icnt[s % 3])) goto out;
        n_roots = sm.bc_a;       // unmatched columns with rows: the first queue segment
        card = p.nc - sm.bc_c;   // all unmatched columns
        iso_free = sm.bc_d;      // unmatched columns without rows (never matchable)
        if (leader) ctl->initial_card = card;
    }
    for (;;) {
        if (n_roots == 0) { no_roots = 1; break; }  // no column left to search from
        if (phases >= p.max_phases) {
            status = p.phase_limit_is_error ? -4 /*BM_ERR_ITER_LIMIT*/ : 1 /*BM_INCOMPLETE*/;
            break;
        }
        ++phases;
        // the phase's endpoint counter (incremental mode: two, alternating by phase,
        // each cleared during the phase before it uses it)
        int32_t* const epc = (incr && (phases & 1) == 0) ? &ctl->ep_alt : &ctl->ep_phase;

        // ---- BFS, level by level (Algorithm 1 inner loop)
        int qb = 0, qe = n_roots, lvl = L0, tail = n_roots;
        if (leader) { ls.levels = 0; ls.first_ep = 0; ls.last_ep = 0; ls.roots_total += n_roots; }
        for (;;) {
            const int s2 = step++;
            if (leader) {
                ctl->qcnt[(s2 + 1) % 3] = 0; ctl->ecnt[(s2 + 1) % 3] = 0; ctl->icnt[(s2 + 1) % 3] = 0; ctl->tcnt[(s2 + 1) % 3] = 0;
                if (DET) ctl->dcnt[(s2 + 1) % 3] = 0;
            }
            if constexpr (DET) step_expand_det(p, qcur, qb, qe, lvl, s2 % 3, cnt, sm);
            else step_expand<WR, RV, true>(p, qcur, qb, qe, lvl, s2 % 3, cnt, sm, p.stamp_base + phases, epc);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, DET ? &ctl->dcnt[s2 % 3] : nullptr)) goto out;
            const int nq = sm.bc_a;           // columns inserted at this level
            const bool found = sm.bc_b > 0;   // some block claimed an endpoint (DET: received an offer)
            if constexpr (DET) {
                if (found) {  // hand the offering rows to their roots
                    const int n_off = sm.bc_c;
                    step_det_offer(p, n_off);
                    if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, nullptr)) goto out;
                    step_det_take(p, n_off, epc);
                    if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, nullptr)) goto out;
                }
            }
            if (leader) {
                const int lv_now = ++ls.levels;
                if (found) {
                    if (ls.first_ep == 0) ls.first_ep = lv_now;
                    ls.last_ep = lv_now;
                }
                ls.ins_total += nq;
            }
            tail = qe + nq;
            if (nq == 0) break;              // no vertex inserted
            if (p.mode == 1 && found) break;  // APsB: stop at the first level with a path
            qb = qe;
            qe += nq;
            ++lvl;
        }
        if (threadIdx.x == 0) sm.bc_c = ld_volatile(epc);  // all appends precede the barrier
        __syncthreads();
        const int n_ep = sm.bc_c;
        if (leader) {
            ls.levels_total += ls.levels;
            if (ls.levels > ls.levels_max) ls.levels_max = ls.levels;
            ls.eps_total += n_ep;
            ctl->n_endpoints_last = n_ep;
            if (p.profile && phases <= p.profile_cap) {
                int32_t* pr = p.profile + 4 * (phases - 1);
                pr[0] = ls.levels;
                pr[1] = n_ep;
                pr[2] = ls.first_ep;
                pr[3] = ls.last_ep;
            }
        }

        if (p.bfs_only) {
            step_release_endpoints(p, n_ep);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, nullptr)) goto out;
            break;
        }
        if (n_ep == 0) break;  // no augmenting path: the matching is maximum (Berge)

        // ---- Alternate (Algorithm 3); the walk is at most as long as the forest
        if (RV && incr) {
            // disjoint walks, and with them the next phase's roots (the roots that took
            // no endpoint), in one step: see step_next_roots
            const int s3 = step++;
            if (leader) {
                ctl->qcnt[(s3 + 1) % 3] = 0; ctl->ecnt[(s3 + 1) % 3] = 0; ctl->icnt[(s3 + 1) % 3] = 0; ctl->tcnt[(s3 + 1) % 3] = 0;
                if (DET) ctl->dcnt[(s3 + 1) % 3] = 0;
                *(epc == &ctl->ep_phase ? &ctl->ep_alt : &ctl->ep_phase) = 0;  // the next phase's counter
            }
            step_alternate_disjoint(p, n_ep, tail + 2);
            step_next_roots<WR, DET, true>(p, qcur, n_roots, tail, qnext, s3 % 3, sm);
        } else {
            step_alternate(p, n_ep, tail + 2, cnt);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, nullptr)) goto out;
            if (incr) {
                const int s3 = step++;
                if (leader) {
                    ctl->qcnt[(s3 + 1) % 3] = 0; ctl->ecnt[(s3 + 1) % 3] = 0; ctl->icnt[(s3 + 1) % 3] = 0; ctl->tcnt[(s3 + 1) % 3] = 0;
                    *(epc == &ctl->ep_phase ? &ctl->ep_alt : &ctl->ep_phase) = 0;  // the next phase's counter
                }
                step_next_roots<WR>(p, qcur, n_roots, tail, qnext, s3 % 3, sm);
            }
        }
        if (incr) {
            // ---- next phase's roots: the unmatched ones among this phase's roots
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, nullptr)) goto out;
            n_roots = sm.bc_a;
#ifdef BM_CHECKED
            step_check_matching(p);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, &ctl->err)) goto out;
            if (sm.bc_c != 0) goto out;
#endif
            card = p.nc - (iso_free + n_roots);
            int2* t = qcur;
            qcur = qnext;
            qnext = t;
        } else {
            // ---- row half of FixMatching, then InitBfsArray (+ column half)
            step_fix_rows(p, cnt);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, nullptr)) goto out;
            const int s = step++;
            if (leader) {
                ctl->qcnt[(s + 1) % 3] = 0; ctl->ecnt[(s + 1) % 3] = 0; ctl->icnt[(s + 1) % 3] = 0; ctl->tcnt[(s + 1) % 3] = 0;
                ctl->ep_phase = 0;
            }
            step_init<WR>(p, qcur, s % 3, cnt, sm);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, &ctl->ecnt[s % 3])) goto out;
            n_roots = sm.bc_a;
            card = p.nc - sm.bc_c;
#ifdef BM_CHECKED
            step_check_matching(p);
            if (!grid_sync(ctl, bid, p.wait_ns, deadline, sm, &ctl->err)) goto out;
            if (sm.bc_c != 0) goto out;
#endif
        }
    }
out:
    flush_counters(p, cnt);
    if (leader) {
        int err = ld_volatile(&ctl->err);
        ctl->status = err != 0 ? err : status;
        ctl->card = card;
        // Algorithm 1's outer iterations: every search, plus the final empty one
        // that Algorithm 1 would run when no column is left to search from
        ctl->phases = phases + no_roots;
        ctl->searches = phases;
        ctl->levels = ls.levels_total;
        ctl->max_levels = ls.levels_max;
        ctl->endpoints = ls.eps_total;
        ctl->inserted = ls.ins_total;
        ctl->roots = ls.roots_total;
        ctl->kernel_ns = (long long)(globaltimer() - ls.t_start);
    }
}

// ---- per-step kernels of the host-driven loop (the paper's structure)
template <bool WR>
__global__ void __launch_bounds__(1024) k_init(Params p, int slot) {
    __shared__ bmd::Smem sm;
    if (threadIdx.x == 0) { sm.qn = 0; sm.npush = 0; sm.has_ep = 0; }
    __syncthreads();
    Counters cnt{0, 0, 0, 0, 0};
    bmd::step_init<WR>(p, p.queue, slot, cnt, sm);
    bmd::flush_counters(p, cnt);
}
template <bool WR>
__global__ void __launch_bounds__(1024) k_expand(Params p, int qb, int qe, int lvl, int slot) {
    __shared__ bmd::Smem sm;
    if (threadIdx.x == 0) { sm.qn = 0; sm.npush = 0; sm.has_ep = 0; }
    __syncthreads();
    Counters cnt{0, 0, 0, 0, 0};
    bmd::step_expand<WR>(p, p.queue, qb, qe, lvl, slot, cnt, sm);
    bmd::flush_counters(p, cnt);
}
__global__ void __launch_bounds__(1024) k_alternate(Params p, int n_ep, int cap) {
    Counters cnt{0, 0, 0, 0, 0};
    bmd::step_alternate(p, n_ep, cap, cnt);
    bmd::flush_counters(p, cnt);
}
__global__ void __launch_bounds__(1024) k_fix(Params p) {
    Counters cnt{0, 0, 0, 0, 0};
    bmd::step_fix_rows(p, cnt);
    bmd::flush_counters(p, cnt);
}
__global__ void __launch_bounds__(1024) k_release(Params p, int n_ep) {
    bmd::step_release_endpoints(p, n_ep);
}

// ---- input checks, greedy, fills
__global__ void k_check_csr(int nr, int nc, long long nnz, const int32_t* __restrict__ cp,
                            const int32_t* __restrict__ ri, Ctl* ctl) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    if (tid == 0 && (cp[0] != 0 || (long long)cp[nc] != nnz)) bad = true;
    for (long long c = tid; c < nc; c += nthr)
        if (cp[c + 1] < cp[c]) bad = true;
    for (long long e = tid; e < nnz; e += nthr) {
        int r = __ldg(&ri[e]);
        if (r < 0 || r >= nr) bad = true;
    }
    if (bad) bmd::set_error(ctl, BM_ERR_INVALID_CSR);
}

__global__ void k_check_matching(int nr, int nc, const int32_t* __restrict__ rm,
                                 const int32_t* __restrict__ cm, Ctl* ctl) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    bool bad = false;
    for (int r = tid; r < nr; r += nthr) {
        int c = rm[r];
        if (c != -1 && (c < 0 || c >= nc || cm[c] != r)) bad = true;
    }
    for (int c = tid; c < nc; c += nthr) {
        int r = cm[c];
        if (r != -1 && (r < 0 || r >= nr || rm[r] != c)) bad = true;
    }
    if (bad) bmd::set_error(ctl, BM_ERR_INVALID_MATCHING);
}

// Installs a matching (rm0/cm0 -> rm/cm) and checks it on the way: every
// entry in range, rm0 and cm0 inverse to each other (BM_ERR_INVALID_MATCHING
// in ctl->err otherwise).  4 entries per thread per pass, their loads in
// flight together; the checks read the source arrays, so nothing waits for
// the copies.
__global__ void k_install_matching(int nr, int nc, const int32_t* __restrict__ rm0,
                                   const int32_t* __restrict__ cm0, int32_t* __restrict__ rm,
                                   int32_t* __restrict__ cm, Ctl* ctl) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    bool bad = false;
    for (int r0 = tid; r0 < nr; r0 += 4 * nthr) {
        int c[4], back[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = r0 + u * nthr < nr ? __ldg(&rm0[r0 + u * nthr]) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) back[u] = (c[u] >= 0 && c[u] < nc) ? __ldg(&cm0[c[u]]) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * nthr;
            if (r >= nr) continue;
            rm[r] = c[u];
            if (c[u] != -1 && (c[u] < 0 || c[u] >= nc || back[u] != r)) bad = true;
        }
    }
    for (int c0 = tid; c0 < nc; c0 += 4 * nthr) {
        int r[4], back[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = c0 + u * nthr < nc ? __ldg(&cm0[c0 + u * nthr]) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) back[u] = (r[u] >= 0 && r[u] < nr) ? __ldg(&rm0[r[u]]) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * nthr;
            if (c >= nc) continue;
            cm[c] = r[u];
            if (r[u] != -1 && (r[u] < 0 || r[u] >= nr || back[u] != c)) bad = true;
        }
    }
    if (bad) bmd::set_error(ctl, BM_ERR_INVALID_MATCHING);
}

__global__ void k_fill(int32_t* a, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

// Cheap matching: each unmatched column claims the first unmatched row of its
// list by CAS.  A column stays unmatched only if all its rows were taken (a
// claim is never given back), so the result is maximal.  Three launches take
// the columns by degree, shortest lists first (a column with few rows has few
// chances, so it chooses before the hubs, which can still find rows far down
// their lists):
//  * light columns (at most GREEDY_LIGHT rows): one thread each, 4 rows per
//    step with the loads in flight together; this pass also lists the medium
//    and heavy columns (R-MAT puts its hubs at neighbouring ids, so the later
//    passes deal them out from these lists instead of by id);
//  * medium columns (up to GREEDY_MEDIUM rows): one warp each, 32 x GREEDY_U
//    rows per step;
//  * heavy columns (R-MAT hubs reach 60,000 rows, most of them taken by then):
//    one block each, blockDim x GREEDY_U rows per step.
// In the cooperative scans every thread loads GREEDY_U rows and their
// matches, the free ones are marked, and their holders try the CAS in list
// order until one wins, so a column still takes the first row of its list
// that was free when it looked.
constexpr int GREEDY_LIGHT = 32;
constexpr int GREEDY_MEDIUM = 2048;
constexpr int GREEDY_U = 4;

struct GreedyLists {
    int32_t* medium;  // [nc] columns of the medium pass
    int32_t* heavy;   // [nc] columns of the heavy pass
    int32_t* count;   // [2] their lengths, zero before the light pass
};

__global__ void k_greedy_light(int nc, const int32_t* __restrict__ cp, const int32_t* __restrict__ ri,
                               int32_t* rm, int32_t* cm, GreedyLists gl, const Ctl* ctl) {
    // after an asynchronous CSR check on the same stream: an invalid CSR is not read
    if (ctl && bmd::ld_volatile(&ctl->err) != 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nc; base += stride) {  // block-uniform
        const int c = (int)(base + threadIdx.x);
        int beg = 0, end = 0;
        if (c < nc && cm[c] == -1) {
            beg = __ldg(&cp[c]);
            end = __ldg(&cp[c + 1]);
        }
        const int deg = end - beg;
        if (deg > GREEDY_MEDIUM) bmd::push(gl.heavy, 0, &gl.count[1], c);
        else if (deg > GREEDY_LIGHT) bmd::push(gl.medium, 0, &gl.count[0], c);
        if (deg > GREEDY_LIGHT) continue;
        bool done = false;
        for (int e = beg; e < end && !done; e += 4) {
            int r[4], m[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) r[u] = e + u < end ? __ldg(&ri[e + u]) : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u) m[u] = r[u] >= 0 ? bmd::ld_volatile(&rm[r[u]]) : 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!done && m[u] == -1 && atomicCAS(&rm[r[u]], -1, c) == -1) {
                    cm[c] = r[u];
                    done = true;
                }
            }
        }
    }
}

__global__ void k_greedy_medium(const int32_t* __restrict__ cp, const int32_t* __restrict__ ri, int32_t* rm,
                                int32_t* cm, GreedyLists gl, const Ctl* ctl) {
    if (ctl && bmd::ld_volatile(&ctl->err) != 0) return;
    const int lane = threadIdx.x & 31;
    const int n = gl.count[0];
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < n; k += nwarps) {  // warp-uniform
        const int hc = gl.medium[k];
        const int hb = __ldg(&cp[hc]), he = __ldg(&cp[hc + 1]);
        bool done = false;
        for (int e0 = hb; e0 < he && !done; e0 += 32 * GREEDY_U) {  // warp-uniform
            int r[GREEDY_U], m[GREEDY_U];
#pragma unroll
            for (int u = 0; u < GREEDY_U; ++u) {
                const int e = e0 + u * 32 + lane;
                r[u] = e < he ? __ldg(&ri[e]) : -1;
            }
#pragma unroll
            for (int u = 0; u < GREEDY_U; ++u) m[u] = r[u] >= 0 ? bmd::ld_volatile(&rm[r[u]]) : 0;
#pragma unroll
            for (int u = 0; u < GREEDY_U; ++u) {
                unsigned free_lanes = __ballot_sync(bmd::FULL, m[u] == -1);
                while (free_lanes && !done) {  // warp-uniform: lowest list position first
                    const int l = __ffs(free_lanes) - 1;
                    free_lanes &= free_lanes - 1;
                    int won = 0;
                    if (lane == l) won = atomicCAS(&rm[r[u]], -1, hc) == -1;
                    won = __shfl_sync(bmd::FULL, won, l);
                    if (won) {
                        if (lane == l) cm[hc] = r[u];
                        done = true;
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(1024) k_greedy_heavy(const int32_t* __restrict__ cp, const int32_t* __restrict__ ri,
                                                       int32_t* rm, int32_t* cm, GreedyLists gl, const Ctl* ctl) {
    if (ctl && bmd::ld_volatile(&ctl->err) != 0) return;
    __shared__ int s_pos, s_done;
    const int T = blockDim.x, t = threadIdx.x;
    const int n = gl.count[1];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {  // block-uniform
        const int hc = gl.heavy[k];
        const int hb = __ldg(&cp[hc]), he = __ldg(&cp[hc + 1]);
        if (t == 0) s_done = 0;
        __syncthreads();
        for (int e0 = hb; e0 < he; e0 += T * GREEDY_U) {  // block-uniform
            int r[GREEDY_U], m[GREEDY_U];
#pragma unroll
            for (int u = 0; u < GREEDY_U; ++u) {
                const int e = e0 + u * T + t;
                r[u] = e < he ? __ldg(&ri[e]) : -1;
            }
#pragma unroll
            for (int u = 0; u < GREEDY_U; ++u) m[u] = r[u] >= 0 ? bmd::ld_volatile(&rm[r[u]]) : 0;
            // window position of this thread's first free row (list order: u major, thread minor)
            int pos = 0x7fffffff;
#pragma unroll
            for (int u = GREEDY_U - 1; u >= 0; --u)
                if (m[u] == -1) pos = u * T + t;
            if (t == 0) s_pos = 0x7fffffff;
            __syncthreads();
            if (pos != 0x7fffffff) atomicMin(&s_pos, pos);
            __syncthreads();
            // candidates in list order; a failed CAS (taken meanwhile) moves on to the next free one
            while (s_pos != 0x7fffffff && !s_done) {  // block-uniform
                const int mypos = s_pos;
                __syncthreads();  // every thread has read s_pos
                if (t == mypos % T) {
                    const int u = mypos / T;
                    int rr = -1;
#pragma unroll
                    for (int v = 0; v < GREEDY_U; ++v)
                        if (v == u) rr = r[v];
                    if (atomicCAS(&rm[rr], -1, hc) == -1) {
                        cm[hc] = rr;
                        s_done = 1;
                    }
                    s_pos = 0x7fffffff;
                }
                __syncthreads();
                if (!s_done) {
                    int next = 0x7fffffff;
#pragma unroll
                    for (int u = GREEDY_U - 1; u >= 0; --u)
                        if (m[u] == -1 && u * T + t > mypos) next = u * T + t;
                    if (next != 0x7fffffff) atomicMin(&s_pos, next);
                }
                __syncthreads();
            }
            if (s_done) break;
        }
        __syncthreads();  // s_done is reset for the next column
    }
}

// The cheap matching (Section 4) on the device: light, medium and heavy
// columns in this order.  `lists` is scratch of 2 x nc int32 (the context's
// queue, free before a match) and `count` two int32 cleared beforehand.
void launch_greedy(int nc, const int32_t* cp, const int32_t* ri, int32_t* rm, int32_t* cm, const Ctl* ctl,
                   int32_t* lists, int32_t* count, int grid, int block, cudaStream_t st) {
    const GreedyLists gl{lists, lists + nc, count};
    k_greedy_light<<<grid, block, 0, st>>>(nc, cp, ri, rm, cm, gl, ctl);
    k_greedy_medium<<<grid, block, 0, st>>>(cp, ri, rm, cm, gl, ctl);
    k_greedy_heavy<<<grid, block, 0, st>>>(cp, ri, rm, cm, gl, ctl);
}

// The cheap matching of the deterministic option over the whole GPU (one
// cooperative launch): rounds in which every unmatched column proposes to the
// first unmatched row of its list and every proposed row takes the smallest
// proposing column (atomicMin in ekey[r]), until a round without proposals.
// Columns of more than 32 rows look for their row a warp at a time, 32 rows
// per step (a ballot of the free ones), from a list built at the start in the
// queue buffer; the others a thread each.  Scratch: level (per column:
// position in its list), root (per column: the row proposed to, -1 none);
// ekey is all ones before and after.
__global__ void __launch_bounds__(1024, 1) k_greedy_rounds(Params p) {
    using namespace bmd;
    __shared__ Smem sm;
    if (threadIdx.x == 0) { sm.qn = 0; sm.npush = 0; sm.has_ep = 0; }
    __syncthreads();
    int bid = 0;
    const unsigned long long deadline = globaltimer() + (unsigned long long)p.total_ns;
    if (ld_volatile(&p.ctl->err) != 0) return;  // CSR check failed before launch
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int warp = tid >> 5, nwarps = nthr >> 5;
    int32_t* pos = p.level;
    int32_t* want = p.root;
    int32_t* longs = (int32_t*)p.queue;
    for (int c = tid; c < p.nc; c += nthr) {
        const int b = __ldg(&p.col_ptr[c]);
        __stcg(&pos[c], b);
        if (__ldg(&p.col_ptr[c + 1]) - b > 32) {
            push(longs, 0, &p.ctl->qcnt[0], c);
            atomicAdd(&sm.npush, 1);
        }
    }
    if (!grid_sync(p.ctl, bid, p.wait_ns, deadline, sm, nullptr)) return;
    const int nlong = sm.bc_a;
    for (int round = 0; round <= p.nc; ++round) {
        bool any = false;
        for (int c = tid; c < p.nc; c += nthr) {  // short lists: a thread each
            const int end = __ldg(&p.col_ptr[c + 1]);
            int at = __ldcg(&pos[c]);
            if (end - __ldg(&p.col_ptr[c]) > 32) continue;
            int w = -1;
            if (__ldcg(&p.cmatch[c]) == -1) {
                while (at < end) {  // 4 rows per step, their matches in flight together
                    int r[4], m[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) r[u] = at + u < end ? __ldg(&p.row_idx[at + u]) : -1;
#pragma unroll
                    for (int u = 0; u < 4; ++u) m[u] = (r[u] >= 0 && idx_ok(p, r[u], p.nr)) ? __ldcg(&p.rmatch[r[u]]) : 0;
                    int k = 0;
                    while (k < 4 && r[k] >= 0 && m[k] != -1) ++k;
                    if (k < 4 && r[k] >= 0) { at += k; w = r[k]; break; }
                    at += 4;
                }
                if (at > end) at = end;
                __stcg(&pos[c], at);
                if (w >= 0) {
                    atomicMin(&p.ekey[w], (unsigned long long)(unsigned)c);
                    any = true;
                }
            }
            __stcg(&want[c], w);
        }
        for (int k = warp; k < nlong; k += nwarps) {  // long lists: a warp each (warp-uniform)
            const int c = __ldcg(&longs[k]);
            if (!idx_ok(p, c, p.nc)) continue;
            int w = -1;
            if (__ldcg(&p.cmatch[c]) == -1) {
                const int end = __ldg(&p.col_ptr[c + 1]);
                int at = __ldcg(&pos[c]);
                while (at < end) {
                    const int r = at + lane < end ? __ldg(&p.row_idx[at + lane]) : -1;
                    const int m = (r >= 0 && idx_ok(p, r, p.nr)) ? __ldcg(&p.rmatch[r]) : 0;
                    const unsigned free_rows = __ballot_sync(FULL, r >= 0 && m == -1);
                    if (free_rows) {
                        const int k0 = __ffs(free_rows) - 1;
                        at += k0;
                        w = __shfl_sync(FULL, r, k0);
                        break;
                    }
                    at += 32;
                }
                if (at > end) at = end;
                if (lane == 0) {
                    __stcg(&pos[c], at);
                    if (w >= 0) atomicMin(&p.ekey[w], (unsigned long long)(unsigned)c);
                }
                if (w >= 0) any = true;
            }
            if (lane == 0) __stcg(&want[c], w);
        }
        if (any) sm.has_ep = 1;
        if (!grid_sync(p.ctl, bid, p.wait_ns, deadline, sm, nullptr)) return;
        const bool more = sm.bc_b > 0;  // some block proposed
        for (int c = tid; c < p.nc; c += nthr) {
            const int w = __ldcg(&want[c]);
            if (w >= 0 && __ldcg(&p.ekey[w]) == (unsigned long long)(unsigned)c) {
                __stcg(&p.rmatch[w], c);
                __stcg(&p.cmatch[c], w);
            }
        }
        if (!grid_sync(p.ctl, bid, p.wait_ns, deadline, sm, nullptr)) return;
        for (int c = tid; c < p.nc; c += nthr) {
            const int w = __ldcg(&want[c]);
            if (w >= 0) __stcg(&p.ekey[w], DKEY_NONE);
        }
        if (!grid_sync(p.ctl, bid, p.wait_ns, deadline, sm, nullptr)) return;
        if (!more) break;
    }
}

__global__ void k_count_matched(int nc, const int32_t* __restrict__ cm, Ctl* ctl) {
    int n = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        n += (cm[c] >= 0);
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) n += __shfl_down_sync(0xffffffffu, n, s);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&ctl->card, n);
}

}  // namespace

// ------------------------------------------------------------------ context
struct bm_ctx {
    int32_t nr = 0, nc = 0;
    int64_t nnz = 0;
    const int32_t* col_ptr = nullptr;
    const int32_t* row_idx = nullptr;
    bool owns_csr = false;
    bool csr_ready = false;
    cudaStream_t stream = nullptr;
    bm_options opt{};
    void* arena = nullptr;  // one device allocation for everything the context owns
    int32_t* rmatch = nullptr;
    int32_t* cmatch = nullptr;
    int32_t* level = nullptr;
    int32_t* root = nullptr;
    int32_t* pred = nullptr;
    int2* queue = nullptr;
    int2* queue2 = nullptr;  // roots of the next phase (one-endpoint GPUBFS-WR)
    int32_t* endpoints = nullptr;
    int32_t* rvis = nullptr;     // per-row claim stamps of the persistent kernel
    int2* crec = nullptr;        // per-column (parent column, matched row) of the last search
    long long stamp_next = 0;    // every stamp in rvis is below stamp_next + 1
    int32_t* profile = nullptr;  // kProfileCap phases x 4
    Ctl* ctl = nullptr;
    Ctl* h_ctl = nullptr;  // pinned mirror
    int32_t sticky = 0;
    int device = 0;
    int num_sms = 0;
    int coop_grid[4] = {0, 0, 0, 0};  // blocks of k_match<false, true>, <true, true>, <true, true, true>;
                                      // k_greedy_rounds
    int block = kDefaultBlock;
    // deterministic option: allocated on its first use, [dkey nc][ekey nr][ecand nr]
    void* det_arena = nullptr;
    unsigned long long* dkey = nullptr;
    unsigned long long* ekey = nullptr;
    int32_t* ecand = nullptr;
};

namespace {

int32_t cuda_fail(bm_ctx* ctx, cudaError_t e) {
    if (e == cudaSuccess) return BM_OK;
    (void)cudaGetLastError();
    if (ctx) ctx->sticky = BM_ERR_CUDA;
    return BM_ERR_CUDA;
}

#define BM_CUDA(ctx, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_); \
    } while (0)

int32_t check_options(const bm_options& o) {
    if (o.mode != BM_APFB && o.mode != BM_APSB) return BM_ERR_INVALID_ARG;
    if (o.bfs != BM_GPUBFS && o.bfs != BM_GPUBFS_WR) return BM_ERR_INVALID_ARG;
    if (o.driver != BM_DRIVER_PERSISTENT && o.driver != BM_DRIVER_HOST) return BM_ERR_INVALID_ARG;
    if (o.max_phases < 0 || o.blocks_per_sm < 0 || o.wait_timeout_ns < 0 || o.total_timeout_ns < 0)
        return BM_ERR_INVALID_ARG;
    if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 1024 || o.block_size % 32 != 0))
        return BM_ERR_INVALID_ARG;
    if (o.deterministic != 0 && o.deterministic != 1) return BM_ERR_INVALID_ARG;
    if (o.deterministic &&
        (o.driver != BM_DRIVER_PERSISTENT || o.bfs != BM_GPUBFS_WR || o.wr_one_endpoint != 1))
        return BM_ERR_INVALID_ARG;
    return BM_OK;
}

int grid_for(bm_ctx* ctx, int n) {  // plain launches: enough blocks to fill the GPU
    long long want = ((long long)n + ctx->block - 1) / ctx->block;
    long long cap = (long long)ctx->num_sms * (2048 / ctx->block);
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

int32_t configure(bm_ctx* ctx) {
    ctx->block = ctx->opt.block_size ? ctx->opt.block_size : kDefaultBlock;
    for (int wr = 0; wr < 4; ++wr) {
        int per_sm = 0;
        cudaError_t e =
            wr == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy_rounds, ctx->block, 0)
            : wr == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<true, true, true>, ctx->block, 0)
            : wr    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<true, true>, ctx->block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<false, true>, ctx->block, 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        int cap = 2048 / ctx->block;  // at most 2048 resident threads per SM
        if (ctx->opt.blocks_per_sm > 0 && ctx->opt.blocks_per_sm < cap) cap = ctx->opt.blocks_per_sm;
        if (per_sm > cap) per_sm = cap;
        while (per_sm > 1 && per_sm * ctx->num_sms > 2047) --per_sm;  // barrier words count blocks in 11 bits
        if (per_sm < 1 || per_sm * ctx->num_sms > 2047) return BM_ERR_UNSUPPORTED;
        ctx->coop_grid[wr] = per_sm * ctx->num_sms;
    }
    return BM_OK;
}

Params make_params(bm_ctx* ctx, bool bfs_only) {
    Params p{};
    p.nr = ctx->nr;
    p.nc = ctx->nc;
    p.col_ptr = ctx->col_ptr;
    p.row_idx = ctx->row_idx;
    p.rmatch = ctx->rmatch;
    p.cmatch = ctx->cmatch;
    p.level = ctx->level;
    p.root = ctx->root;
    p.pred = ctx->pred;
    p.queue = ctx->queue;
    p.queue2 = ctx->queue2;
    p.endpoints = ctx->endpoints;
    p.rvis = ctx->rvis;
    p.crec = ctx->crec;
    p.ctl = ctx->ctl;
    p.mode = ctx->opt.mode;
    p.one_ep = ctx->opt.wr_one_endpoint;
    const int safety = (ctx->nr < ctx->nc ? ctx->nr : ctx->nc) + 2;
    if (bfs_only) {
        p.max_phases = 1;
        p.phase_limit_is_error = 0;
    } else if (ctx->opt.max_phases > 0 && ctx->opt.max_phases < safety) {
        p.max_phases = ctx->opt.max_phases;
        p.phase_limit_is_error = 0;
    } else {
        p.max_phases = safety;
        p.phase_limit_is_error = 1;
    }
    p.bfs_only = bfs_only ? 1 : 0;
    p.profile = ctx->profile;
    p.profile_cap = kProfileCap;
    p.chk = &ctx->ctl->err;
    p.wait_ns = ctx->opt.wait_timeout_ns ? ctx->opt.wait_timeout_ns : 5000000000LL;
    p.total_ns = ctx->opt.total_timeout_ns ? ctx->opt.total_timeout_ns : 120000000000LL;
    return p;
}

int32_t validate_csr_async(bm_ctx* ctx) {
    const long long work = ctx->nnz > ctx->nc ? ctx->nnz : (long long)ctx->nc + 1;
    const int g = grid_for(ctx, (int)(work < (1 << 30) ? work : (1 << 30)));
    k_check_csr<<<g, ctx->block, 0, ctx->stream>>>(ctx->nr, ctx->nc, ctx->nnz, ctx->col_ptr, ctx->row_idx, ctx->ctl);
    BM_CUDA(ctx, cudaGetLastError());
    return BM_OK;
}

int32_t sync_ctl(bm_ctx* ctx) {
    BM_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    BM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return BM_OK;
}

// Host-driven Algorithm 1: one launch per step; the host reads the step
// counters after every BFS level, as the paper's host loop reads its flags.
template <bool WR>
int32_t run_host_loop(bm_ctx* ctx, const Params& p) {
    Ctl* h = ctx->h_ctl;
    const int gb = grid_for(ctx, ctx->nc > ctx->nr ? ctx->nc : ctx->nr);
    const int blk = ctx->block;
    cudaStream_t st = ctx->stream;
    int phases = 0, card = 0, status = 0, no_roots = 0;
    long long levels_total = 0, levels_max = 0, eps_total = 0, ins_total = 0, roots_total = 0;
    int step = 0;
    auto clear_slot = [&](int slot) -> int32_t {
        BM_CUDA(ctx, cudaMemsetAsync(&ctx->ctl->qcnt[slot], 0, sizeof(int32_t), st));
        BM_CUDA(ctx, cudaMemsetAsync(&ctx->ctl->ecnt[slot], 0, sizeof(int32_t), st));
        BM_CUDA(ctx, cudaMemsetAsync(&ctx->ctl->tcnt[slot], 0, sizeof(int32_t), st));
        return BM_OK;
    };
    auto clear_phase = [&]() -> int32_t {
        BM_CUDA(ctx, cudaMemsetAsync(&ctx->ctl->ep_phase, 0, sizeof(int32_t), st));
        return BM_OK;
    };
    int32_t rc = sync_ctl(ctx);
    if (rc) return rc;
    if (h->err) return h->err;
    for (;;) {
        int s = step++;
        if ((rc = clear_slot(s % 3))) return rc;
        if ((rc = clear_phase())) return rc;
        k_init<WR><<<gb, blk, 0, st>>>(p, s % 3);
        BM_CUDA(ctx, cudaGetLastError());
        if ((rc = sync_ctl(ctx))) return rc;
        const int n_roots = h->qcnt[s % 3];
        card = p.nc - h->ecnt[s % 3];
        if (phases == 0) {
            BM_CUDA(ctx, cudaMemcpyAsync(&ctx->ctl->initial_card, &card, sizeof(int), cudaMemcpyHostToDevice, st));
        }
        if (n_roots == 0) { no_roots = 1; break; }
        if (phases >= p.max_phases) { status = p.phase_limit_is_error ? BM_ERR_ITER_LIMIT : BM_INCOMPLETE; break; }
        ++phases;
        roots_total += n_roots;
        int qb = 0, qe = n_roots, lvl = L0, n_ep = 0, levels = 0, first_ep = 0, last_ep = 0;
        for (;;) {
            int s2 = step++;
            if ((rc = clear_slot(s2 % 3))) return rc;
            const int g = grid_for(ctx, qe - qb);
            k_expand<WR><<<g, blk, 0, st>>>(p, qb, qe, lvl, s2 % 3);
            BM_CUDA(ctx, cudaGetLastError());
            if ((rc = sync_ctl(ctx))) return rc;
            const int nq = h->qcnt[s2 % 3];
            const int new_ep = h->ep_phase - n_ep;
            n_ep = h->ep_phase;
            ++levels;
            if (new_ep > 0) {
                if (first_ep == 0) first_ep = levels;
                last_ep = levels;
            }
            ins_total += nq;
            if (nq == 0) break;
            if (p.mode == BM_APSB && n_ep > 0) break;
            if (levels > p.nc + 2) return BM_ERR_ITER_LIMIT;
            qb = qe;
            qe += nq;
            ++lvl;
        }
        levels_total += levels;
        if (levels > levels_max) levels_max = levels;
        eps_total += n_ep;
        if (phases <= p.profile_cap) {
            int32_t rec[4] = {levels, n_ep, first_ep, last_ep};
            BM_CUDA(ctx, cudaMemcpyAsync(p.profile + 4 * (phases - 1), rec, sizeof(rec), cudaMemcpyHostToDevice, st));
            BM_CUDA(ctx, cudaStreamSynchronize(st));
        }
        if (p.bfs_only) {
            if (n_ep) k_release<<<grid_for(ctx, n_ep), blk, 0, st>>>(p, n_ep);
            BM_CUDA(ctx, cudaGetLastError());
            BM_CUDA(ctx, cudaMemcpyAsync(&ctx->ctl->n_endpoints_last, &n_ep, sizeof(int), cudaMemcpyHostToDevice, st));
            break;
        }
        if (n_ep == 0) break;
        k_alternate<<<grid_for(ctx, n_ep), blk, 0, st>>>(p, n_ep, levels + 2);
        BM_CUDA(ctx, cudaGetLastError());
        k_fix<<<grid_for(ctx, p.nr), blk, 0, st>>>(p);
        BM_CUDA(ctx, cudaGetLastError());
    }
    if ((rc = sync_ctl(ctx))) return rc;
    Ctl fin = *h;
    fin.status = fin.err ? fin.err : status;
    fin.card = card;
    fin.phases = phases + no_roots;
    fin.searches = phases;
    fin.roots = roots_total;
    fin.levels = levels_total;
    fin.max_levels = levels_max;
    fin.endpoints = eps_total;
    fin.inserted = ins_total;
    BM_CUDA(ctx, cudaMemcpyAsync(ctx->ctl, &fin, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    return sync_ctl(ctx);
}

// The deterministic option's arrays, allocated on first use: [dkey nc][ekey nr][ecand nr].
int32_t ensure_det_arena(bm_ctx* ctx) {
    if (ctx->det_arena) return BM_OK;
    const size_t nr1 = (size_t)(ctx->nr ? ctx->nr : 1), nc1 = (size_t)(ctx->nc ? ctx->nc : 1);
    const size_t off_ek = (8 * nc1 + 255) & ~size_t(255);
    const size_t off_ec = off_ek + ((8 * nr1 + 255) & ~size_t(255));
    if (cudaMalloc(&ctx->det_arena, off_ec + 4 * nr1) != cudaSuccess) {
        (void)cudaGetLastError();
        ctx->det_arena = nullptr;
        return BM_ERR_NOMEM;
    }
    char* a = (char*)ctx->det_arena;
    ctx->dkey = (unsigned long long*)a;
    ctx->ekey = (unsigned long long*)(a + off_ek);
    ctx->ecand = (int32_t*)(a + off_ec);
    return BM_OK;
}

// Runs the method (or one BFS) on the installed matching.  The control block
// is cleared by the caller beforehand so that input checks queued before can
// report through it.
int32_t run(bm_ctx* ctx, bool bfs_only) {
    Params p = make_params(ctx, bfs_only);
    const bool wr = ctx->opt.bfs == BM_GPUBFS_WR;
    if (ctx->opt.driver == BM_DRIVER_HOST) {
        int32_t rc = wr ? run_host_loop<true>(ctx, p) : run_host_loop<false>(ctx, p);
        if (rc < 0 && ctx->sticky == 0) ctx->sticky = rc;
        return rc < 0 ? rc : ctx->h_ctl->status;
    }
    // row stamps of this launch: stamp_next + 1 ... stamp_next + max_phases; the
    // array is cleared when they would pass INT32_MAX
    const long long span = (long long)p.max_phases + 1;
    if (ctx->stamp_next + span >= 0x7fffffffLL) {
        BM_CUDA(ctx, cudaMemsetAsync(ctx->rvis, 0, 4 * (size_t)(ctx->nr ? ctx->nr : 1), ctx->stream));
        ctx->stamp_next = 0;
    }
    p.stamp_base = (int32_t)ctx->stamp_next;
    ctx->stamp_next += span;
    void* args[] = {&p};
    if (ctx->opt.deterministic) {
        int32_t rc = ensure_det_arena(ctx);
        if (rc) return rc;
        // every key "none" (all ones) at launch; the kernel restores that between phases
        BM_CUDA(ctx, cudaMemsetAsync(ctx->det_arena, 0xff, (size_t)((char*)ctx->ecand - (char*)ctx->det_arena),
                                     ctx->stream));
        p.dkey = ctx->dkey;
        p.ekey = ctx->ekey;
        p.ecand = ctx->ecand;
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_match<true, true, true>, ctx->coop_grid[2],
                                                    ctx->block, args, 0, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        return BM_OK;
    }
    cudaError_t e = wr ? cudaLaunchCooperativeKernel((const void*)k_match<true, true>, ctx->coop_grid[1], ctx->block, args, 0, ctx->stream)
                       : cudaLaunchCooperativeKernel((const void*)k_match<false, true>, ctx->coop_grid[0], ctx->block, args, 0, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    return BM_OK;
}

int32_t finish(bm_ctx* ctx, int32_t* card_out, bm_stats* stats) {
    int32_t rc = sync_ctl(ctx);
    if (rc) return rc;
    const Ctl& h = *ctx->h_ctl;
    const int32_t status = h.status != 0 ? h.status : h.err;
    if (status < 0) ctx->sticky = status;
    if (card_out) *card_out = h.card;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->status = status;
        stats->phases = h.phases;
        stats->initial_card = h.initial_card;
        stats->final_card = h.card;
        stats->levels = h.levels;
        stats->max_levels_in_phase = h.max_levels;
        stats->columns_expanded = h.cols_expanded;
        stats->edges_scanned = h.edges_scanned;
        stats->endpoints = h.endpoints;
        stats->fix_repairs = h.fix_repairs;
        stats->inserted = h.inserted;
        stats->edges_to_matched = h.edges_matched;
        stats->alternate_steps = h.alt_steps;
        stats->kernel_ns = h.kernel_ns;
        stats->roots = h.roots;
        if (ctx->opt.driver == BM_DRIVER_PERSISTENT) {
            stats->grid = ctx->coop_grid[ctx->opt.deterministic ? 2 : ctx->opt.bfs == BM_GPUBFS_WR ? 1 : 0];
            stats->block = ctx->block;
        }
    }
    return status;
}

}  // namespace

// ------------------------------------------------------------------ C-ABI
extern "C" {

void bm_default_options(bm_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->mode = BM_APFB;
    opt->bfs = BM_GPUBFS_WR;
    opt->driver = BM_DRIVER_PERSISTENT;
    opt->wr_one_endpoint = 1;
}

int32_t bm_version(void) { return kVersion; }

const char* bm_status_string(int32_t s) {
    switch (s) {
        case BM_OK: return "ok";
        case BM_INCOMPLETE: return "phase limit reached (matching valid, maybe not maximum)";
        case BM_ERR_INVALID_ARG: return "invalid argument";
        case BM_ERR_INVALID_CSR: return "invalid CSR (col_ptr not monotone from 0 to nnz, or row id out of range)";
        case BM_ERR_NOMEM: return "out of device or pinned memory";
        case BM_ERR_ITER_LIMIT: return "safety cap on phases, levels or walk length reached";
        case BM_ERR_TIMEOUT: return "device-side barrier wait timed out";
        case BM_ERR_CUDA: return "CUDA runtime error";
        case BM_ERR_STATE: return "context in error state or call out of order";
        case BM_ERR_UNSUPPORTED: return "device cannot run the cooperative launch";
        case BM_ERR_INVALID_MATCHING: return "initial matching out of range or rmatch/cmatch not inverse";
        case BM_ERR_TOO_LARGE: return "graph too large for the allocation-free entry point's scratch";
        case BM_ERR_CHECK: return "range-checked build: an index out of range or an inconsistent matching";
        default: return "unknown status";
    }
}

int32_t bm_create(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* col_ptr,
                  const int32_t* row_idx, void* stream, const bm_options* opt, bm_ctx** out) {
    bmi::NvtxRange nvtx_range("bm_create");
    if (!out) return BM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL) return BM_ERR_INVALID_ARG;
    if (col_ptr == nullptr && row_idx != nullptr) return BM_ERR_INVALID_ARG;
    if (col_ptr != nullptr && row_idx == nullptr && nnz > 0) return BM_ERR_INVALID_ARG;
    bm_options o;
    if (opt) o = *opt; else bm_default_options(&o);
    int32_t rc = check_options(o);
    if (rc) return rc;

    bm_ctx* ctx = new (std::nothrow) bm_ctx();
    if (!ctx) return BM_ERR_NOMEM;
    ctx->nr = n_rows;
    ctx->nc = n_cols;
    ctx->nnz = nnz;
    ctx->stream = (cudaStream_t)stream;
    ctx->opt = o;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return BM_ERR_CUDA;
    }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (!coop) { delete ctx; return BM_ERR_UNSUPPORTED; }

    // arena: [ctl][rmatch nr][cmatch nc][level nc][root nc][pred nr][queue nc][queue2 nc][endpoints nr]
    //        [rvis nr][crec nc][profile][csr?]
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t nr1 = (size_t)(n_rows ? n_rows : 1), nc1 = (size_t)(n_cols ? n_cols : 1);
    size_t off_ctl = 0;
    size_t off_rm = off_ctl + al(sizeof(Ctl));
    size_t off_cm = off_rm + al(4 * nr1);
    size_t off_lv = off_cm + al(4 * nc1);
    size_t off_rt = off_lv + al(4 * nc1);
    size_t off_pd = off_rt + al(4 * nc1);
    size_t off_q = off_pd + al(4 * nr1);
    size_t off_q2 = off_q + al(8 * nc1);
    size_t off_ep = off_q2 + al(8 * nc1);
    size_t off_rv = off_ep + al(4 * nr1);
    size_t off_cr = off_rv + al(4 * nr1);
    size_t off_pf = off_cr + al(8 * nc1);
    size_t off_cp = off_pf + al(4 * 4 * (size_t)kProfileCap);
    size_t total = off_cp;
    const bool own = (col_ptr == nullptr);
    size_t off_ri = 0;
    if (own) {
        off_ri = off_cp + al(4 * ((size_t)n_cols + 1));
        total = off_ri + al(4 * (size_t)(nnz ? nnz : 1));
    }
    if (cudaMalloc(&ctx->arena, total) != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return BM_ERR_NOMEM;
    }
    if (cudaMallocHost((void**)&ctx->h_ctl, sizeof(Ctl)) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(ctx->arena);
        delete ctx;
        return BM_ERR_NOMEM;
    }
    char* a = (char*)ctx->arena;
    ctx->ctl = (Ctl*)(a + off_ctl);
    ctx->rmatch = (int32_t*)(a + off_rm);
    ctx->cmatch = (int32_t*)(a + off_cm);
    ctx->level = (int32_t*)(a + off_lv);
    ctx->root = (int32_t*)(a + off_rt);
    ctx->pred = (int32_t*)(a + off_pd);
    ctx->queue = (int2*)(a + off_q);
    ctx->queue2 = (int2*)(a + off_q2);
    ctx->endpoints = (int32_t*)(a + off_ep);
    ctx->rvis = (int32_t*)(a + off_rv);
    ctx->crec = (int2*)(a + off_cr);
    ctx->profile = (int32_t*)(a + off_pf);
    if (own) {
        ctx->owns_csr = true;
        ctx->col_ptr = (int32_t*)(a + off_cp);
        ctx->row_idx = (int32_t*)(a + off_ri);
    } else {
        ctx->col_ptr = col_ptr;
        ctx->row_idx = row_idx;
    }
    rc = configure(ctx);
    if (rc) { bm_destroy(ctx); return rc; }
    cudaStream_t st = ctx->stream;
    if (cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st) != cudaSuccess ||
        cudaMemsetAsync(ctx->rmatch, 0xff, 4 * nr1, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->cmatch, 0xff, 4 * nc1, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->pred, 0xff, 4 * nr1, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->rvis, 0, 4 * nr1, st) != cudaSuccess) {
        cuda_fail(ctx, cudaGetLastError());
        bm_destroy(ctx);
        return BM_ERR_CUDA;
    }
    if (!own) {
        rc = validate_csr_async(ctx);
        if (!rc) rc = sync_ctl(ctx);
        if (!rc && ctx->h_ctl->err) rc = ctx->h_ctl->err;
        if (rc) { bm_destroy(ctx); return rc; }
        ctx->csr_ready = true;
    } else {
        rc = sync_ctl(ctx);
        if (rc) { bm_destroy(ctx); return rc; }
    }
    *out = ctx;
    return BM_OK;
}

int32_t bm_set_options(bm_ctx* ctx, const bm_options* opt) {
    if (!ctx || !opt) return BM_ERR_INVALID_ARG;
    if (ctx->sticky) return BM_ERR_STATE;
    int32_t rc = check_options(*opt);
    if (rc) return rc;
    ctx->opt = *opt;
    return configure(ctx);
}

int32_t bm_upload_csr(bm_ctx* ctx, const int32_t* h_col_ptr, const int32_t* h_row_idx) {
    bmi::NvtxRange nvtx_range("bm_upload_csr");
    if (!ctx || !h_col_ptr || (!h_row_idx && ctx->nnz > 0)) return BM_ERR_INVALID_ARG;
    if (ctx->sticky || !ctx->owns_csr) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    BM_CUDA(ctx, cudaMemcpyAsync((void*)ctx->col_ptr, h_col_ptr, 4 * ((size_t)ctx->nc + 1), cudaMemcpyHostToDevice, st));
    if (ctx->nnz)
        BM_CUDA(ctx, cudaMemcpyAsync((void*)ctx->row_idx, h_row_idx, 4 * (size_t)ctx->nnz, cudaMemcpyHostToDevice, st));
    int32_t rc = validate_csr_async(ctx);
    if (!rc) rc = sync_ctl(ctx);
    if (rc) return rc;
    if (ctx->h_ctl->err) { ctx->csr_ready = false; return ctx->h_ctl->err; }
    ctx->csr_ready = true;
    return BM_OK;
}

int32_t bm_greedy(bm_ctx* ctx, int32_t* card_out) {
    bmi::NvtxRange nvtx_range("bm_greedy");
    if (!ctx) return BM_ERR_INVALID_ARG;
    if (ctx->sticky || !ctx->csr_ready) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    if (ctx->nc && ctx->opt.deterministic) {
        // proposal rounds: the same matching on every run and launch geometry
        int32_t rc = ensure_det_arena(ctx);
        if (rc) return rc;
        BM_CUDA(ctx, cudaMemsetAsync(ctx->ekey, 0xff, 8 * (size_t)(ctx->nr ? ctx->nr : 1), st));
        Params p = make_params(ctx, false);
        p.ekey = ctx->ekey;
        void* args[] = {&p};
        BM_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_greedy_rounds, ctx->coop_grid[3], ctx->block, args, 0, st));
        k_count_matched<<<grid_for(ctx, ctx->nc), ctx->block, 0, st>>>(ctx->nc, ctx->cmatch, ctx->ctl);
        BM_CUDA(ctx, cudaGetLastError());
    } else if (ctx->nc) {
        launch_greedy(ctx->nc, ctx->col_ptr, ctx->row_idx, ctx->rmatch, ctx->cmatch, nullptr, (int32_t*)ctx->queue,
                      &ctx->ctl->qcnt[0], grid_for(ctx, ctx->nc), ctx->block, st);
        BM_CUDA(ctx, cudaGetLastError());
        k_count_matched<<<grid_for(ctx, ctx->nc), ctx->block, 0, st>>>(ctx->nc, ctx->cmatch, ctx->ctl);
        BM_CUDA(ctx, cudaGetLastError());
    }
    int32_t rc = sync_ctl(ctx);
    if (rc) return rc;
    if (ctx->h_ctl->err) {  // a barrier wait of the rounds ran out of time
        ctx->sticky = ctx->h_ctl->err;
        return ctx->h_ctl->err;
    }
    if (card_out) *card_out = ctx->h_ctl->card;
    return BM_OK;
}

int32_t bm_set_matching(bm_ctx* ctx, const int32_t* rmatch, const int32_t* cmatch) {
    bmi::NvtxRange nvtx_range("bm_set_matching");
    if (!ctx || ((rmatch == nullptr) != (cmatch == nullptr))) return BM_ERR_INVALID_ARG;
    if (ctx->sticky) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    if (!rmatch) {
        BM_CUDA(ctx, cudaMemsetAsync(ctx->rmatch, 0xff, 4 * (size_t)ctx->nr, st));
        BM_CUDA(ctx, cudaMemsetAsync(ctx->cmatch, 0xff, 4 * (size_t)ctx->nc, st));
        return BM_OK;
    }
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    if (ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(ctx->rmatch, rmatch, 4 * (size_t)ctx->nr, cudaMemcpyDeviceToDevice, st));
    if (ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(ctx->cmatch, cmatch, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToDevice, st));
    k_check_matching<<<grid_for(ctx, ctx->nr > ctx->nc ? ctx->nr : ctx->nc), ctx->block, 0, st>>>(ctx->nr, ctx->nc, ctx->rmatch, ctx->cmatch, ctx->ctl);
    BM_CUDA(ctx, cudaGetLastError());
    int32_t rc = sync_ctl(ctx);
    if (rc) return rc;
    if (ctx->h_ctl->err) {
        // leave a valid (empty) matching installed
        cudaMemsetAsync(ctx->rmatch, 0xff, 4 * (size_t)ctx->nr, st);
        cudaMemsetAsync(ctx->cmatch, 0xff, 4 * (size_t)ctx->nc, st);
        cudaStreamSynchronize(st);
        return ctx->h_ctl->err;
    }
    return BM_OK;
}

int32_t bm_get_matching(bm_ctx* ctx, int32_t* rmatch_out, int32_t* cmatch_out) {
    if (!ctx) return BM_ERR_INVALID_ARG;
    if (ctx->sticky) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    if (rmatch_out && ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(rmatch_out, ctx->rmatch, 4 * (size_t)ctx->nr, cudaMemcpyDeviceToDevice, st));
    if (cmatch_out && ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(cmatch_out, ctx->cmatch, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToDevice, st));
    BM_CUDA(ctx, cudaStreamSynchronize(st));
    return BM_OK;
}

int32_t bm_match(bm_ctx* ctx, int32_t* rmatch_out, int32_t* cmatch_out, int32_t* card_out, bm_stats* stats) {
    bmi::NvtxRange nvtx_range("bm_match");
    if (!ctx) return BM_ERR_INVALID_ARG;
    if (ctx->sticky || !ctx->csr_ready) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    int32_t rc = run(ctx, false);
    if (rc < 0) return rc;
    if (rmatch_out && ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(rmatch_out, ctx->rmatch, 4 * (size_t)ctx->nr, cudaMemcpyDeviceToDevice, st));
    if (cmatch_out && ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(cmatch_out, ctx->cmatch, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToDevice, st));
    return finish(ctx, card_out, stats);
}

int32_t bm_match_from(bm_ctx* ctx, const int32_t* rmatch0, const int32_t* cmatch0, int32_t* rmatch_out,
                      int32_t* cmatch_out, int32_t* card_out, bm_stats* stats) {
    bmi::NvtxRange nvtx_range("bm_match_from");
    if (!ctx || !rmatch0 || !cmatch0) return BM_ERR_INVALID_ARG;
    if (ctx->sticky || !ctx->csr_ready) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    // copy and check in one launch; the check reports through the control block, and the
    // match launch then returns at once
    k_install_matching<<<grid_for(ctx, ((ctx->nr > ctx->nc ? ctx->nr : ctx->nc) + 3) / 4), ctx->block, 0, st>>>(
        ctx->nr, ctx->nc, rmatch0, cmatch0, ctx->rmatch, ctx->cmatch, ctx->ctl);
    BM_CUDA(ctx, cudaGetLastError());
    int32_t rc = run(ctx, false);
    if (rc < 0) return rc;
    if (rmatch_out && ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(rmatch_out, ctx->rmatch, 4 * (size_t)ctx->nr, cudaMemcpyDeviceToDevice, st));
    if (cmatch_out && ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(cmatch_out, ctx->cmatch, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToDevice, st));
    rc = finish(ctx, card_out, stats);
    if (rc == BM_ERR_INVALID_MATCHING) {
        ctx->sticky = 0;  // bad input is not a broken context: leave the empty matching installed
        cudaMemsetAsync(ctx->rmatch, 0xff, 4 * (size_t)ctx->nr, st);
        cudaMemsetAsync(ctx->cmatch, 0xff, 4 * (size_t)ctx->nc, st);
        cudaStreamSynchronize(st);
    }
    return rc;
}

int32_t bm_match_host(bm_ctx* ctx, const int32_t* h_col_ptr, const int32_t* h_row_idx,
                      int32_t* h_rmatch, int32_t* h_cmatch, int32_t* card_out, bm_stats* stats) {
    bmi::NvtxRange nvtx_range("bm_match_host");
    if (!ctx || !h_col_ptr || (!h_row_idx && ctx->nnz > 0) || ((h_rmatch == nullptr) != (h_cmatch == nullptr)))
        return BM_ERR_INVALID_ARG;
    if (ctx->sticky || !ctx->owns_csr) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    BM_CUDA(ctx, cudaMemcpyAsync((void*)ctx->col_ptr, h_col_ptr, 4 * ((size_t)ctx->nc + 1), cudaMemcpyHostToDevice, st));
    if (ctx->nnz)
        BM_CUDA(ctx, cudaMemcpyAsync((void*)ctx->row_idx, h_row_idx, 4 * (size_t)ctx->nnz, cudaMemcpyHostToDevice, st));
    if (h_rmatch) {
        if (ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(ctx->rmatch, h_rmatch, 4 * (size_t)ctx->nr, cudaMemcpyHostToDevice, st));
        if (ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(ctx->cmatch, h_cmatch, 4 * (size_t)ctx->nc, cudaMemcpyHostToDevice, st));
    } else {
        BM_CUDA(ctx, cudaMemsetAsync(ctx->rmatch, 0xff, 4 * (size_t)ctx->nr, st));
        BM_CUDA(ctx, cudaMemsetAsync(ctx->cmatch, 0xff, 4 * (size_t)ctx->nc, st));
    }
    // input checks report through the control block; the match launch then
    // returns at once if one failed
    int32_t rc = validate_csr_async(ctx);
    if (rc) return rc;
    k_check_matching<<<grid_for(ctx, ctx->nr > ctx->nc ? ctx->nr : ctx->nc), ctx->block, 0, st>>>(ctx->nr, ctx->nc, ctx->rmatch, ctx->cmatch, ctx->ctl);
    BM_CUDA(ctx, cudaGetLastError());
    ctx->csr_ready = true;
    if (ctx->opt.driver == BM_DRIVER_HOST) {
        rc = sync_ctl(ctx);
        if (rc) return rc;
        if (ctx->h_ctl->err) { ctx->csr_ready = false; return ctx->h_ctl->err; }
    }
    rc = run(ctx, false);
    if (rc < 0) return rc;
    if (h_rmatch) {
        if (ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(h_rmatch, ctx->rmatch, 4 * (size_t)ctx->nr, cudaMemcpyDeviceToHost, st));
        if (ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(h_cmatch, ctx->cmatch, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToHost, st));
    }
    rc = finish(ctx, card_out, stats);
    if (rc == BM_ERR_INVALID_CSR || rc == BM_ERR_INVALID_MATCHING) {
        ctx->csr_ready = false;
        ctx->sticky = 0;  // bad input is not a broken context
        cudaMemsetAsync(ctx->rmatch, 0xff, 4 * (size_t)ctx->nr, st);
        cudaMemsetAsync(ctx->cmatch, 0xff, 4 * (size_t)ctx->nc, st);
        cudaStreamSynchronize(st);
    }
    return rc;
}

int32_t bm_bfs(bm_ctx* ctx, int32_t* level_out, int32_t* root_out, int32_t* pred_out,
               int32_t* endpoints_out, int32_t* n_endpoints_out) {
    bmi::NvtxRange nvtx_range("bm_bfs");
    if (!ctx) return BM_ERR_INVALID_ARG;
    if (ctx->sticky || !ctx->csr_ready) return BM_ERR_STATE;
    cudaStream_t st = ctx->stream;
    BM_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st));
    BM_CUDA(ctx, cudaMemsetAsync(ctx->pred, 0xff, 4 * (size_t)(ctx->nr ? ctx->nr : 1), st));
    if (ctx->opt.bfs != BM_GPUBFS_WR && ctx->nc) {
        k_fill<<<grid_for(ctx, ctx->nc), ctx->block, 0, st>>>(ctx->root, ctx->nc, -1);
        BM_CUDA(ctx, cudaGetLastError());
    }
    int32_t rc = run(ctx, true);
    if (rc < 0) return rc;
    rc = sync_ctl(ctx);
    if (rc) return rc;
    const int n_ep = ctx->h_ctl->n_endpoints_last;
    if (level_out && ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(level_out, ctx->level, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToDevice, st));
    if (root_out && ctx->nc) BM_CUDA(ctx, cudaMemcpyAsync(root_out, ctx->root, 4 * (size_t)ctx->nc, cudaMemcpyDeviceToDevice, st));
    if (pred_out && ctx->nr) BM_CUDA(ctx, cudaMemcpyAsync(pred_out, ctx->pred, 4 * (size_t)ctx->nr, cudaMemcpyDeviceToDevice, st));
    if (endpoints_out && n_ep) BM_CUDA(ctx, cudaMemcpyAsync(endpoints_out, ctx->endpoints, 4 * (size_t)n_ep, cudaMemcpyDeviceToDevice, st));
    if (n_endpoints_out) *n_endpoints_out = n_ep;
    rc = finish(ctx, nullptr, nullptr);
    return rc == BM_INCOMPLETE ? BM_OK : rc;
}

int32_t bm_phase_profile(bm_ctx* ctx, int32_t cap, int32_t* levels, int32_t* endpoints,
                         int32_t* first_ep_level, int32_t* last_ep_level, int32_t* n_out) {
    if (!ctx || cap < 0 || !n_out) return BM_ERR_INVALID_ARG;
    if (ctx->sticky) return BM_ERR_STATE;
    int32_t rc = sync_ctl(ctx);
    if (rc) return rc;
    int n = ctx->h_ctl->searches;  // phases that searched with at least one root
    if (n > kProfileCap) n = kProfileCap;
    if (n > cap) n = cap;
    *n_out = n;
    if (n == 0) return BM_OK;
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)n);
    if (!tmp) return BM_ERR_NOMEM;
    cudaError_t e = cudaMemcpyAsync(tmp, ctx->profile, sizeof(int32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { free(tmp); return cuda_fail(ctx, e); }
    for (int i = 0; i < n; ++i) {
        if (levels) levels[i] = tmp[4 * i];
        if (endpoints) endpoints[i] = tmp[4 * i + 1];
        if (first_ep_level) first_ep_level[i] = tmp[4 * i + 2];
        if (last_ep_level) last_ep_level[i] = tmp[4 * i + 3];
    }
    free(tmp);
    return BM_OK;
}

int32_t bm_destroy(bm_ctx* ctx) {
    if (!ctx) return BM_ERR_INVALID_ARG;
    if (ctx->stream || ctx->arena) cudaStreamSynchronize(ctx->stream);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->det_arena) cudaFree(ctx->det_arena);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    (void)cudaGetLastError();
    delete ctx;
    return BM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free entry point
// For callers that may not allocate device memory (see bm_match_noalloc in
// bmatch.h): the working arrays of the matching kernel live in this fixed
// file-scope array instead of a context's allocation.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

struct NoallocDevice {
    bool ready;
    unsigned char* scratch;  // device address of g_noalloc_scratch on this device
    int grid;                // cooperative grid of k_match<true, false>
    int block;
    int sms;
};
NoallocDevice g_noalloc_dev[kMaxDevices];
std::mutex g_noalloc_mutex;

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// The control block's share of the scratch array: a fixed size, so that the
// size limit stated in bmatch.h does not move when the control block grows.
constexpr size_t kNoallocCtlBytes = 1024;
static_assert(sizeof(Ctl) <= kNoallocCtlBytes, "control block outgrew its share of the scratch array");

// Once per device, with that device current: the host-side name of the array
// is not a device address, so look the address up and keep it.
int32_t noalloc_setup(int dev, NoallocDevice* out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
        int sms = 0, coop = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<true, false>, kDefaultBlock, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            return BM_ERR_CUDA;
        }
        if (!coop || per_sm < 1) return BM_ERR_UNSUPPORTED;
        if (per_sm > 2048 / kDefaultBlock) per_sm = 2048 / kDefaultBlock;
        while (per_sm > 1 && per_sm * sms > 2047) --per_sm;  // barrier words count blocks in 11 bits
        if (per_sm * sms > 2047) return BM_ERR_UNSUPPORTED;
        d.scratch = (unsigned char*)ptr;
        d.grid = per_sm * sms;
        d.block = kDefaultBlock;
        d.sms = sms;
        d.ready = true;
    }
    *out = d;
    return BM_OK;
}

}  // namespace

extern "C" int32_t bm_match_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                    const int32_t* col_ptr, const int32_t* row_idx,
                                    int32_t* rmatch, int32_t* cmatch, void* stream,
                                    int32_t* card_out) {
    bmi::NvtxRange nvtx_range("bm_match_noalloc");
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL) return BM_ERR_INVALID_ARG;
    if (!col_ptr || (!row_idx && nnz > 0) || (!rmatch && n_rows > 0) || (!cmatch && n_cols > 0))
        return BM_ERR_INVALID_ARG;
    const size_t nr = (size_t)n_rows, nc = (size_t)n_cols;
    const size_t off_lv = kNoallocCtlBytes;
    const size_t off_rt = off_lv + round256(4 * nc);
    const size_t off_pd = off_rt + round256(4 * nc);
    const size_t off_q = off_pd + round256(4 * nr);
    const size_t off_ep = off_q + round256(8 * nc);
    const size_t need = off_ep + round256(4 * nr);
    if (need > (size_t)BM_NOALLOC_SCRATCH_BYTES) return BM_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return BM_ERR_UNSUPPORTED;
    NoallocDevice d;
    int32_t rc = noalloc_setup(dev, &d);
    if (rc) return rc;

    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* s = d.scratch;
    Ctl* ctl = (Ctl*)s;
    Params p{};
    p.nr = n_rows;
    p.nc = n_cols;
    p.col_ptr = col_ptr;
    p.row_idx = row_idx;
    p.rmatch = rmatch;
    p.cmatch = cmatch;
    p.level = (int32_t*)(s + off_lv);
    p.root = (int32_t*)(s + off_rt);
    p.pred = (int32_t*)(s + off_pd);
    p.queue = (int2*)(s + off_q);
    p.endpoints = (int32_t*)(s + off_ep);
    p.ctl = ctl;
    p.chk = &ctl->err;
    p.mode = BM_APFB;
    p.one_ep = 1;
    p.max_phases = (n_rows < n_cols ? n_rows : n_cols) + 2;
    p.phase_limit_is_error = 1;
    p.bfs_only = 0;
    p.wait_ns = 5000000000LL;
    p.total_ns = 120000000000LL;

    // the control block (barrier counter, step counters, error word) must start at zero;
    // the other arrays are written before they are read
    if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) != cudaSuccess) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
    const int threads = 2048 / d.block * d.sms;
    const long long work = nnz > n_cols ? nnz : (long long)n_cols + 1;
    int g = (int)((work + d.block - 1) / d.block);
    if (g > threads) g = threads;
    if (g < 1) g = 1;
    k_check_csr<<<g, d.block, 0, st>>>(n_rows, n_cols, nnz, col_ptr, row_idx, ctl);
    const int n_max = n_rows > n_cols ? n_rows : n_cols;
    int g2 = (n_max + d.block - 1) / d.block;
    if (g2 > threads) g2 = threads;
    if (g2 < 1) g2 = 1;
    k_check_matching<<<g2, d.block, 0, st>>>(n_rows, n_cols, rmatch, cmatch, ctl);
    if (cudaGetLastError() != cudaSuccess) return BM_ERR_CUDA;
    void* args[] = {&p};
    if (cudaLaunchCooperativeKernel((const void*)k_match<true, false>, d.grid, d.block, args, 0, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return BM_ERR_CUDA;
    }
    Ctl h;  // pageable host copy of the control block
    if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return BM_ERR_CUDA;
    }
    const int32_t status = h.status != 0 ? h.status : h.err;
    if (card_out) *card_out = h.card;
    return status;
}

// ------------------------------------------------------------------ internal: whole-GPU match of one graph
namespace {
struct ExclusiveDevice {
    bool ready;
    int grid[4];  // cooperative grid of k_match<false, true>, <true, true>, <true, true, true>; k_greedy_rounds
    int sms;
};
ExclusiveDevice g_excl_dev[kMaxDevices];
std::mutex g_excl_mutex;
}  // namespace

int32_t bmi::enqueue_match(bmd::Params p, long long nnz, bool wr, int greedy, cudaStream_t st, int blocks_per_sm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return BM_ERR_UNSUPPORTED;
    ExclusiveDevice d;
    {
        std::lock_guard<std::mutex> lock(g_excl_mutex);
        ExclusiveDevice& e = g_excl_dev[dev];
        if (!e.ready) {
            int sms = 0, coop = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
                (void)cudaGetLastError();
                return BM_ERR_CUDA;
            }
            if (!coop) return BM_ERR_UNSUPPORTED;
            for (int w = 0; w < 4; ++w) {
                int per_sm = 0;
                const cudaError_t r =
                    w == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy_rounds, kDefaultBlock, 0)
                    : w == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<true, true, true>, kDefaultBlock, 0)
                    : w ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<true, true>, kDefaultBlock, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<false, true>, kDefaultBlock, 0);
                if (r != cudaSuccess) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
                if (per_sm > 2048 / kDefaultBlock) per_sm = 2048 / kDefaultBlock;
                while (per_sm > 1 && per_sm * sms > 2047) --per_sm;  // barrier words count blocks in 11 bits
                if (per_sm < 1 || per_sm * sms > 2047) return BM_ERR_UNSUPPORTED;
                e.grid[w] = per_sm * sms;
            }
            e.sms = sms;
            e.ready = true;
        }
        d = e;
    }
    const int B = kDefaultBlock;
    const int threads = 2048 / B * d.sms;
    auto grid_of = [&](long long n) {
        long long g = (n + B - 1) / B;
        if (g > threads) g = threads;
        return (int)(g < 1 ? 1 : g);
    };
    const size_t nr = (size_t)p.nr, nc = (size_t)p.nc;
    if (cudaMemsetAsync(p.ctl, 0, sizeof(Ctl), st) != cudaSuccess) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
    k_check_csr<<<grid_of(nnz > p.nc ? nnz : (long long)p.nc + 1), B, 0, st>>>(p.nr, p.nc, nnz, p.col_ptr,
                                                                               p.row_idx, p.ctl);
    if ((nr && (cudaMemsetAsync(p.rmatch, 0xff, 4 * nr, st) != cudaSuccess ||
                cudaMemsetAsync(p.rvis, 0, 4 * nr, st) != cudaSuccess)) ||
        (nc && cudaMemsetAsync(p.cmatch, 0xff, 4 * nc, st) != cudaSuccess)) {
        (void)cudaGetLastError();
        return BM_ERR_CUDA;
    }
    const bool det = p.dkey != nullptr;  // deterministic option (GPUBFS-WR, one endpoint per root)
    auto cap = [&](int g) { return (blocks_per_sm > 0 && g > blocks_per_sm * d.sms) ? blocks_per_sm * d.sms : g; };
    if (det && ((nc && cudaMemsetAsync(p.dkey, 0xff, 8 * nc, st) != cudaSuccess) ||
                (nr && cudaMemsetAsync(p.ekey, 0xff, 8 * nr, st) != cudaSuccess))) {
        (void)cudaGetLastError();
        return BM_ERR_CUDA;
    }
    if (greedy && det) {
        // proposal rounds; their barrier words and list count are cleared for the matching
        // kernel afterwards (the error word, set by the CSR check, stays)
        if (p.wait_ns <= 0) p.wait_ns = 5000000000LL;
        if (p.total_ns <= 0) p.total_ns = 120000000000LL;
        void* gargs[] = {&p};
        if (cudaLaunchCooperativeKernel((const void*)k_greedy_rounds, cap(d.grid[3]), B, gargs, 0, st) != cudaSuccess ||
            cudaMemsetAsync(&p.ctl->arrive[0][0], 0, sizeof(p.ctl->arrive), st) != cudaSuccess ||
            cudaMemsetAsync(&p.ctl->qcnt[0], 0, 2 * sizeof(int32_t), st) != cudaSuccess) {
            (void)cudaGetLastError();
            return BM_ERR_CUDA;
        }
    } else if (greedy) {
        // the cheap matching counts its lists in the control block's first two queue
        // counters, which the matching kernel needs at zero
        launch_greedy(p.nc, p.col_ptr, p.row_idx, p.rmatch, p.cmatch, p.ctl, (int32_t*)p.queue, &p.ctl->qcnt[0],
                      grid_of(p.nc), B, st);
        if (cudaMemsetAsync(&p.ctl->qcnt[0], 0, 2 * sizeof(int32_t), st) != cudaSuccess) {
            (void)cudaGetLastError();
            return BM_ERR_CUDA;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return BM_ERR_CUDA;
    p.bfs_only = 0;
    p.profile = nullptr;
    p.profile_cap = 0;
    p.chk = &p.ctl->err;
    p.max_phases = (p.nr < p.nc ? p.nr : p.nc) + 2;
    p.phase_limit_is_error = 1;
    p.stamp_base = 0;  // the stamps were just cleared
    if (p.wait_ns <= 0) p.wait_ns = 5000000000LL;
    if (p.total_ns <= 0) p.total_ns = 120000000000LL;
    void* args[] = {&p};
    const int grid = cap(d.grid[det ? 2 : wr ? 1 : 0]);
    const cudaError_t e = det  ? cudaLaunchCooperativeKernel((const void*)k_match<true, true, true>, grid, B, args, 0, st)
                          : wr ? cudaLaunchCooperativeKernel((const void*)k_match<true, true>, grid, B, args, 0, st)
                               : cudaLaunchCooperativeKernel((const void*)k_match<false, true>, grid, B, args, 0, st);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return BM_ERR_CUDA; }
    return BM_OK;
}
