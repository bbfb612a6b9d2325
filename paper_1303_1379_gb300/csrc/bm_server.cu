// Continuous-batching matching server.
//
// Requests (host CSR graphs) arrive at any time.  A host scheduler thread
// admits them in arrival order when their device memory fits in a fixed pool
// and a ring slot is free, uploads the CSR on a copy stream, and publishes a
// descriptor to a ring in host-mapped memory.  A persistent worker kernel
// (one block per request at a time, blocks independent of each other) polls
// the ring, claims the next published request with a CAS on a device counter,
// validates and matches it (cheap matching + Algorithm 1 of arXiv 1303.1379,
// the same block routine as the batched path) and writes |M| and a done flag
// back to host-mapped memory.  So requests that arrive while others run are
// picked up by whichever block frees first: their work overlaps on the GPU.
// Workers leave after an idle period (every wait is bounded) and the
// scheduler relaunches them when work is published.
// A request with at least exclusive_min_edges edges would hold one block for
// tens of milliseconds; it runs on the single-graph persistent kernel
// instead.  By default (exclusive_alongside) that launch shares the GPU with
// the workers: the workers keep one block per SM and the large requests run
// one after another on their own stream with one block per SM, so both stay
// resident and small requests do not queue behind large ones.  Otherwise the
// workers are told to leave (they finish the requests they hold), the checks,
// the cheap matching and the launch are queued behind them on the same
// stream, consecutive large requests run back to back behind one departure,
// and the next request for the workers waits until they are done (arrival
// order).
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bm_device.cuh"
#include "bm_internal.h"
#include "bm_pool.h"
#include "bmatch.h"

using bmd::Counters;
using bmd::Params;
using bmd::Smem;
using bms::PoolAllocator;

namespace {

// Descriptor of a published request (host-mapped; written by the host before
// the request is published, read by the worker that claims it).
struct SlotDesc {
    long long id;
    long long nnz;
    long long off_cp, off_ri, off_rm, off_cm, off_lv, off_rt, off_q, off_pd, off_ep;  // bytes into the pool
    long long off_dk, off_ek, off_ec;  // deterministic option's keys and offer list
    int32_t nr, nc;
    int32_t greedy;
    int32_t pad;
};
// Completion record (host-mapped; written by the worker).
struct SlotDone {
    int32_t done;  // ticket + 1 once finished
    int32_t card;
    int32_t status;
    int32_t phases;
    long long levels;
};
struct alignas(128) MappedHead {
    long long published;  // tickets published so far
    int32_t stop;         // workers leave when set
    int32_t pad[27];
};

struct ServeParams {
    unsigned char* pool;
    const MappedHead* head;  // device view of host-mapped memory
    const SlotDesc* desc;
    SlotDone* done;
    unsigned long long* claimed;  // device memory: tickets claimed so far
    int32_t* busy;                // device memory: blocks working on a request
    int32_t ring;
    int32_t mode, one_ep;
    int32_t pad;
    long long idle_ns;
};

__device__ __forceinline__ long long ld_acquire_sys_s64(const long long* p) {
    long long v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_sys_s32(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_sys_s64(const long long* p) {
    long long v;
    asm volatile("ld.relaxed.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_sys_s32(int32_t* p, int v) {
    asm volatile("st.relaxed.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys_s32(int32_t* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// DET: every request with the deterministic option's rules
// (block_match_graph_det).
template <bool WR, bool DET = false>
__global__ void __launch_bounds__(1024, 1) k_serve(ServeParams sp) {
    __shared__ Smem sm;
    __shared__ unsigned s_vis[bmd::SB_MAX_COLS / 32], s_srv[bmd::SB_MAX_COLS / 32];  // see block_match_graph
    __shared__ long long s_ticket;
    __shared__ SlotDesc s_d;
    Counters cnt{0, 0, 0, 0, 0};
    unsigned long long idle0 = bmd::globaltimer();
    for (;;) {
        __syncthreads();  // s_ticket / s_d of the previous round have been read
        if (threadIdx.x == 0) {
            // Poll for work with exponential back-off.  A block leaves only when
            // no block has been busy for idle_ns, so the workers stay together
            // while any request runs and leave together when the server idles.
            long long t = -1;
            unsigned sleep_ns = 128;
            for (int spin = 0; spin < 64 && t == -1; ++spin) {
                if (ld_relaxed_sys_s32(&sp.head->stop)) { t = -2; break; }
                const long long pub = ld_acquire_sys_s64(&sp.head->published);
                const unsigned long long c = *(volatile unsigned long long*)sp.claimed;
                if ((long long)c < pub) {
                    if (atomicCAS(sp.claimed, c, c + 1) == c) {
                        t = (long long)c;
                        atomicAdd(sp.busy, 1);
                    }
                    continue;
                }
                const unsigned long long now = bmd::globaltimer();
                if (bmd::ld_volatile(sp.busy) > 0) idle0 = now;
                if (now - idle0 > (unsigned long long)sp.idle_ns) { t = -2; break; }
                __nanosleep(sleep_ns);
                if (sleep_ns < 16384) sleep_ns <<= 1;
            }
            s_ticket = t;
            if (t >= 0) {
                const SlotDesc* d = &sp.desc[t % sp.ring];
                s_d.id = ld_relaxed_sys_s64(&d->id);
                s_d.nnz = ld_relaxed_sys_s64(&d->nnz);
                s_d.off_cp = ld_relaxed_sys_s64(&d->off_cp);
                s_d.off_ri = ld_relaxed_sys_s64(&d->off_ri);
                s_d.off_rm = ld_relaxed_sys_s64(&d->off_rm);
                s_d.off_cm = ld_relaxed_sys_s64(&d->off_cm);
                s_d.off_lv = ld_relaxed_sys_s64(&d->off_lv);
                s_d.off_rt = ld_relaxed_sys_s64(&d->off_rt);
                s_d.off_q = ld_relaxed_sys_s64(&d->off_q);
                s_d.off_pd = ld_relaxed_sys_s64(&d->off_pd);
                s_d.off_ep = ld_relaxed_sys_s64(&d->off_ep);
                if (DET) {
                    s_d.off_dk = ld_relaxed_sys_s64(&d->off_dk);
                    s_d.off_ek = ld_relaxed_sys_s64(&d->off_ek);
                    s_d.off_ec = ld_relaxed_sys_s64(&d->off_ec);
                }
                s_d.nr = ld_relaxed_sys_s32(&d->nr);
                s_d.nc = ld_relaxed_sys_s32(&d->nc);
                s_d.greedy = ld_relaxed_sys_s32(&d->greedy);
            }
        }
        __syncthreads();
        const long long t = s_ticket;
        if (t == -2) break;
        if (t == -1) continue;
        if (threadIdx.x == 0) idle0 = bmd::globaltimer();
        Params p{};
        p.nr = s_d.nr;
        p.nc = s_d.nc;
        p.col_ptr = (const int32_t*)(sp.pool + s_d.off_cp);
        p.row_idx = (const int32_t*)(sp.pool + s_d.off_ri);
        p.rmatch = (int32_t*)(sp.pool + s_d.off_rm);
        p.cmatch = (int32_t*)(sp.pool + s_d.off_cm);
        p.level = (int32_t*)(sp.pool + s_d.off_lv);
        p.root = (int32_t*)(sp.pool + s_d.off_rt);
        p.queue = (int2*)(sp.pool + s_d.off_q);
        p.pred = (int32_t*)(sp.pool + s_d.off_pd);
        p.endpoints = (int32_t*)(sp.pool + s_d.off_ep);
        p.mode = sp.mode;
        p.one_ep = sp.one_ep;
        int card = 0, phases = 0, status = 0;
        long long levels = 0, eps = 0, ins = 0;
        // the CSR came from the host: check it before any indexed read
        if (!bmd::block_check_csr<false>(p.nr, p.nc, s_d.nnz, p.col_ptr, p.row_idx, sm)) {
            status = BM_ERR_INVALID_CSR;
        } else {
            for (int r = threadIdx.x; r < p.nr; r += blockDim.x) __stcg(&p.rmatch[r], -1);
            for (int c = threadIdx.x; c < p.nc; c += blockDim.x) __stcg(&p.cmatch[c], -1);
            __syncthreads();
            if constexpr (DET) {
                p.dkey = (unsigned long long*)(sp.pool + s_d.off_dk);
                p.ekey = (unsigned long long*)(sp.pool + s_d.off_ek);
                p.ecand = (int32_t*)(sp.pool + s_d.off_ec);
                if (p.nc <= bmd::SB_MAX_COLS) {  // visited marks in shared memory
                    p.vis = s_vis;
                    status = bmd::block_match_graph_det<false, true>(p, s_d.greedy, sm, cnt, card, phases, levels,
                                                                     eps, ins);
                } else {
                    status = bmd::block_match_graph_det<false>(p, s_d.greedy, sm, cnt, card, phases, levels, eps,
                                                               ins);
                }
            } else if (WR && sp.one_ep && p.nc <= bmd::SB_MAX_COLS) {  // tree marks in shared memory
                p.vis = s_vis;
                p.srv = s_srv;
                status = bmd::block_match_graph<WR, false, false, WR>(p, s_d.greedy, sm, cnt, card, phases, levels,
                                                                        eps, ins);
            } else {
                status = bmd::block_match_graph<WR, false>(p, s_d.greedy, sm, cnt, card, phases, levels, eps, ins);
            }
        }
        if (threadIdx.x == 0) {
            SlotDone* d = &sp.done[t % sp.ring];
            st_relaxed_sys_s32(&d->card, card);
            st_relaxed_sys_s32(&d->status, status);
            st_relaxed_sys_s32(&d->phases, phases);
            __threadfence_system();
            st_release_sys_s32(&d->done, (int)(t + 1));
            atomicSub(sp.busy, 1);
            idle0 = bmd::globaltimer();
        }
    }
}


enum ReqState { PENDING = 0, UPLOADING = 1, RUNNING = 2, DONE = 3, CANCELLED = 4 };

struct Request {
    long long id = 0;
    int32_t nr = 0, nc = 0;
    long long nnz = 0;
    const int32_t* h_cp = nullptr;
    const int32_t* h_ri = nullptr;
    int32_t greedy = 1;
    int state = PENDING;
    size_t off = 0, bytes = 0;
    bool has_mem = false;
    long long ticket = -1;
    cudaEvent_t uploaded = nullptr;
    int32_t card = 0, status = 0, phases = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
    size_t off_rm = 0, off_cm = 0;
};

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int kOffs = 16;      // arrays of a request's pool region
constexpr int kExclSlots = 64;  // whole-GPU runs queued at once

// A request's region: its CSR, matching and the workspace of the worker
// routine (offsets 0-8); requests with at least exclusive_min_edges edges also
// get the rest of a whole-GPU launch's workspace (9-12); with the
// deterministic option, the keys and the offer list (13-15).
size_t request_bytes(int32_t nr, int32_t nc, long long nnz, bool exclusive, bool det, size_t* offs) {
    const size_t NR = (size_t)(nr ? nr : 1), NC = (size_t)(nc ? nc : 1);
    size_t o = 0;
    offs[0] = o; o += round256(4 * ((size_t)nc + 1));       // col_ptr
    offs[1] = o; o += round256(4 * (size_t)(nnz ? nnz : 1));  // row_idx
    offs[2] = o; o += round256(4 * NR);                       // rmatch
    offs[3] = o; o += round256(4 * NC);                       // cmatch
    offs[4] = o; o += round256(4 * NC);                       // level
    offs[5] = o; o += round256(4 * NC);                       // root
    offs[6] = o; o += round256(8 * NC);                       // queue
    offs[7] = o; o += round256(4 * NR);                       // pred
    offs[8] = o; o += round256(4 * NR);                       // endpoints
    offs[9] = offs[10] = offs[11] = offs[12] = o;
    if (exclusive) {
        offs[9] = o; o += round256(8 * NC);                   // queue2
        offs[10] = o; o += round256(4 * NR);                  // claim stamps
        offs[11] = o; o += round256(8 * NC);                  // Alternate records
        offs[12] = o; o += round256(sizeof(bmd::Ctl));        // control block
    }
    offs[13] = offs[14] = offs[15] = o;
    if (det) {
        offs[13] = o; o += round256(8 * NC);                  // tree-entry keys
        offs[14] = o; o += round256(8 * NR);                  // offer keys
        offs[15] = o; o += round256(4 * NR);                  // rows offered during a level
    }
    return o;
}

}  // namespace

struct bm_server {
    bm_server_options opt{};
    int device = 0;
    int num_sms = 0;
    int block = 512;
    int grid = 0;
    cudaStream_t copy_stream = nullptr;
    cudaStream_t work_stream = nullptr;
    cudaStream_t excl_stream = nullptr;  // whole-GPU runs that share the GPU with the workers
    unsigned char* pool = nullptr;
    PoolAllocator* alloc = nullptr;
    void* mapped = nullptr;  // host-mapped: head, desc[ring], done[ring]
    MappedHead* head = nullptr;
    SlotDesc* desc = nullptr;
    SlotDone* done = nullptr;
    void* d_mapped = nullptr;  // device view
    unsigned long long* d_claimed = nullptr;
    int32_t* d_busy = nullptr;
    cudaEvent_t worker_ev = nullptr;
    bool worker_launched = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<long long> pending;
    std::deque<long long> uploading;
    std::unordered_map<long long, Request> reqs;
    std::vector<long long> ring_owner;  // request id per ring slot, -1 if free
    // requests running alone on the whole GPU, in launch order: (request id, slot of
    // excl_ev / h_excl_ctl).  Consecutive ones run back to back behind one departure
    // of the workers.
    std::deque<std::pair<long long, int>> excl_runs;
    std::vector<int> excl_free;            // free slots
    cudaEvent_t excl_ev[kExclSlots] = {};  // recorded after a launch and the copy of its control block
    bmd::Ctl* h_excl_ctl = nullptr;        // pinned copies of the control blocks [kExclSlots]
    long long exclusive_runs = 0;
    long long next_id = 1;
    long long next_ticket = 0;
    int inflight = 0;  // uploading + running
    long long completed = 0, rejected = 0, launches = 0;
    int32_t sticky = 0;
    std::atomic<bool> running{false};
    std::thread sched;
};

namespace {

void launch_workers(bm_server* s) {
    ServeParams sp{};
    sp.pool = s->pool;
    char* dm = (char*)s->d_mapped;
    sp.head = (const MappedHead*)dm;
    sp.desc = (const SlotDesc*)(dm + sizeof(MappedHead));
    sp.done = (SlotDone*)(dm + sizeof(MappedHead) + sizeof(SlotDesc) * (size_t)s->opt.ring_slots);
    sp.claimed = s->d_claimed;
    sp.busy = s->d_busy;
    sp.ring = s->opt.ring_slots;
    sp.mode = s->opt.mode;
    sp.one_ep = 1;
    sp.idle_ns = s->opt.idle_timeout_ns;
    if (s->opt.deterministic) k_serve<true, true><<<s->grid, s->block, 0, s->work_stream>>>(sp);
    else if (s->opt.bfs == BM_GPUBFS_WR) k_serve<true><<<s->grid, s->block, 0, s->work_stream>>>(sp);
    else k_serve<false><<<s->grid, s->block, 0, s->work_stream>>>(sp);
    if (cudaGetLastError() != cudaSuccess) { s->sticky = BM_ERR_CUDA; return; }
    cudaEventRecord(s->worker_ev, s->work_stream);
    s->worker_launched = true;
    s->launches++;
}

// A request large enough to run alone on the whole GPU (the persistent
// single-graph kernel) rather than on one worker block.
bool is_exclusive(const bm_server* s, const Request& r) {
    return s->opt.exclusive_min_edges > 0 && r.nnz >= s->opt.exclusive_min_edges;
}

// Starts request r alone on the whole GPU: the workers are told to leave, and
// the whole-GPU launch is queued behind them on the work stream, followed by
// the copy of its control block and an event.  Returns BM_OK or an error.
int32_t start_exclusive(bm_server* s, Request& r, int slot) {
    size_t offs[kOffs];
    request_bytes(r.nr, r.nc, r.nnz, true, s->opt.deterministic != 0, offs);
    unsigned char* b = s->pool + r.off;
    bmd::Params p{};
    p.nr = r.nr;
    p.nc = r.nc;
    p.col_ptr = (const int32_t*)(b + offs[0]);
    p.row_idx = (const int32_t*)(b + offs[1]);
    p.rmatch = (int32_t*)(b + offs[2]);
    p.cmatch = (int32_t*)(b + offs[3]);
    p.level = (int32_t*)(b + offs[4]);
    p.root = (int32_t*)(b + offs[5]);
    p.queue = (int2*)(b + offs[6]);
    p.pred = (int32_t*)(b + offs[7]);
    p.endpoints = (int32_t*)(b + offs[8]);
    p.queue2 = (int2*)(b + offs[9]);
    p.rvis = (int32_t*)(b + offs[10]);
    p.crec = (int2*)(b + offs[11]);
    p.ctl = (bmd::Ctl*)(b + offs[12]);
    if (s->opt.deterministic) {  // the same rules as the workers: the same result on either lane
        p.dkey = (unsigned long long*)(b + offs[13]);
        p.ekey = (unsigned long long*)(b + offs[14]);
        p.ecand = (int32_t*)(b + offs[15]);
    }
    p.mode = s->opt.mode;
    p.one_ep = 1;
    // alongside: the launch takes one block per SM beside the workers' one, on its own
    // stream; otherwise the workers finish what they hold and leave first
    const bool along = s->opt.exclusive_alongside != 0;
    if (!along) __atomic_store_n(&s->head->stop, 1, __ATOMIC_RELEASE);
    cudaStream_t st = along ? s->excl_stream : s->work_stream;
    int32_t rc = bmi::enqueue_match(p, r.nnz, s->opt.bfs == BM_GPUBFS_WR, r.greedy, st, along ? 1 : 0);
    if (rc != BM_OK) return rc;
    if (cudaMemcpyAsync(&s->h_excl_ctl[slot], p.ctl, sizeof(bmd::Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(s->excl_ev[slot], st) != cudaSuccess) {
        (void)cudaGetLastError();
        return BM_ERR_CUDA;
    }
    return BM_OK;
}

// One scheduling pass; called with s->mu held.  Returns whether anything moved.
bool schedule_once(bm_server* s) {
    bool moved = false;
    const int ring = s->opt.ring_slots;
    // completions
    for (int k = 0; k < ring; ++k) {
        const long long id = s->ring_owner[k];
        if (id < 0) continue;
        Request& r = s->reqs[id];
        const int d = __atomic_load_n(&s->done[k].done, __ATOMIC_ACQUIRE);
        if (d != (int)(r.ticket + 1)) continue;
        r.card = s->done[k].card;
        r.status = s->done[k].status;
        r.phases = s->done[k].phases;
        r.state = DONE;
        r.t_done = std::chrono::steady_clock::now();
        s->ring_owner[k] = -1;
        s->inflight--;
        s->completed++;
        if (!s->opt.keep_results && r.has_mem) { s->alloc->release(r.off, r.bytes); r.has_mem = false; }
        moved = true;
    }
    // requests running alone: finished, in launch order?
    while (!s->excl_runs.empty()) {
        const long long id = s->excl_runs.front().first;
        const int slot = s->excl_runs.front().second;
        const cudaError_t q = cudaEventQuery(s->excl_ev[slot]);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) { (void)cudaGetLastError(); s->sticky = BM_ERR_CUDA; break; }
        Request& r = s->reqs[id];
        const bmd::Ctl& h = s->h_excl_ctl[slot];
        r.card = h.card;
        r.status = h.status != 0 ? h.status : h.err;
        r.phases = h.phases;
        r.state = DONE;
        r.t_done = std::chrono::steady_clock::now();
        s->inflight--;
        s->completed++;
        if (!s->opt.keep_results && r.has_mem) { s->alloc->release(r.off, r.bytes); r.has_mem = false; }
        s->excl_runs.pop_front();
        s->excl_free.push_back(slot);
        moved = true;
    }
    // with no whole-GPU run queued the workers may run (again); starting one sets stop
    if (s->excl_runs.empty() && !s->opt.exclusive_alongside) __atomic_store_n(&s->head->stop, 0, __ATOMIC_RELEASE);
    // uploads that finished, in order: publish to the workers, or run alone; a
    // request for the workers waits until the whole-GPU runs ahead of it are done
    while (!s->uploading.empty()) {
        Request& r = s->reqs[s->uploading.front()];
        const cudaError_t q = cudaEventQuery(r.uploaded);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) { s->sticky = BM_ERR_CUDA; break; }
        if (is_exclusive(s, r)) {
            if (s->excl_free.empty()) break;
            const int slot = s->excl_free.back();
            const int32_t rc = start_exclusive(s, r, slot);
            if (rc != BM_OK) { s->sticky = rc; break; }
            s->excl_free.pop_back();
            s->excl_runs.emplace_back(r.id, slot);
            r.state = RUNNING;
            s->exclusive_runs++;
            s->uploading.pop_front();
            moved = true;
            continue;
        }
        if (!s->excl_runs.empty() && !s->opt.exclusive_alongside) break;
        const int slot = (int)(s->next_ticket % ring);
        if (s->ring_owner[slot] != -1) break;  // ticket next_ticket - ring still running
        const long long ticket = s->next_ticket++;
        size_t offs[kOffs];
        request_bytes(r.nr, r.nc, r.nnz, false, s->opt.deterministic != 0, offs);
        SlotDesc& d = s->desc[slot];
        d.id = r.id;
        d.nnz = r.nnz;
        d.off_cp = (long long)(r.off + offs[0]);
        d.off_ri = (long long)(r.off + offs[1]);
        d.off_rm = (long long)(r.off + offs[2]);
        d.off_cm = (long long)(r.off + offs[3]);
        d.off_lv = (long long)(r.off + offs[4]);
        d.off_rt = (long long)(r.off + offs[5]);
        d.off_q = (long long)(r.off + offs[6]);
        d.off_pd = (long long)(r.off + offs[7]);
        d.off_ep = (long long)(r.off + offs[8]);
        d.off_dk = (long long)(r.off + offs[13]);
        d.off_ek = (long long)(r.off + offs[14]);
        d.off_ec = (long long)(r.off + offs[15]);
        d.nr = r.nr;
        d.nc = r.nc;
        d.greedy = r.greedy;
        r.ticket = ticket;
        r.state = RUNNING;
        s->ring_owner[slot] = r.id;
        __atomic_store_n(&s->head->published, ticket + 1, __ATOMIC_RELEASE);
        s->uploading.pop_front();
        moved = true;
    }
    // admissions, in arrival order
    while (!s->pending.empty() && s->inflight < ring) {
        const long long id = s->pending.front();
        Request& r = s->reqs[id];
        if (r.state == CANCELLED) { s->pending.pop_front(); continue; }
        size_t offs[kOffs];
        r.bytes = request_bytes(r.nr, r.nc, r.nnz, is_exclusive(s, r), s->opt.deterministic != 0, offs);
        if (r.bytes > s->alloc->size()) {  // can never fit
            r.state = DONE;
            r.status = BM_ERR_TOO_LARGE;
            r.t_done = std::chrono::steady_clock::now();
            s->rejected++;
            s->pending.pop_front();
            moved = true;
            continue;
        }
        size_t off = 0;
        if (!s->alloc->alloc(r.bytes, &off)) break;  // wait for memory to free up
        r.off = off;
        r.has_mem = true;
        r.off_rm = off + offs[2];
        r.off_cm = off + offs[3];
        cudaMemcpyAsync(s->pool + off + offs[0], r.h_cp, 4 * ((size_t)r.nc + 1), cudaMemcpyHostToDevice, s->copy_stream);
        if (r.nnz) cudaMemcpyAsync(s->pool + off + offs[1], r.h_ri, 4 * (size_t)r.nnz, cudaMemcpyHostToDevice, s->copy_stream);
        if (!r.uploaded) cudaEventCreateWithFlags(&r.uploaded, cudaEventDisableTiming);
        cudaEventRecord(r.uploaded, s->copy_stream);
        if (cudaGetLastError() != cudaSuccess) { s->sticky = BM_ERR_CUDA; break; }
        r.state = UPLOADING;
        s->inflight++;
        s->uploading.push_back(id);
        s->pending.pop_front();
        moved = true;
    }
    // workers: keep one launch alive while requests are published (not while one runs alone)
    bool need = false;
    for (int k = 0; k < ring && !need; ++k) need = s->ring_owner[k] >= 0 && s->reqs[s->ring_owner[k]].state == RUNNING;
    if (need && (s->excl_runs.empty() || s->opt.exclusive_alongside)) {
        const bool alive = s->worker_launched && cudaEventQuery(s->worker_ev) == cudaErrorNotReady;
        if (!alive) launch_workers(s);
    }
    return moved;
}

void scheduler_main(bm_server* s) {
    cudaSetDevice(s->device);
    while (s->running.load()) {
        bool moved;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            moved = schedule_once(s);
        }
        if (moved) s->cv.notify_all();
        else std::this_thread::sleep_for(std::chrono::microseconds(s->opt.poll_interval_us));
    }
}

}  // namespace

extern "C" {

void bm_server_default_options(bm_server_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->pool_bytes = 0;
    o->reserve_bytes = 2ll << 30;
    o->ring_slots = 1024;
    o->block_size = 512;
    o->blocks_per_sm = 2;
    o->mode = BM_APFB;
    o->bfs = BM_GPUBFS_WR;
    o->keep_results = 0;
    o->idle_timeout_ns = 50000000;  // 50 ms
    o->poll_interval_us = 5;
    o->exclusive_min_edges = 1 << 19;
    o->exclusive_alongside = 1;
}

int32_t bm_server_create(const bm_server_options* opt, bm_server** out) {
    if (!out) return BM_ERR_INVALID_ARG;
    *out = nullptr;
    bm_server_options o;
    if (opt) o = *opt; else bm_server_default_options(&o);
    if (o.ring_slots < 1 || o.ring_slots > (1 << 20) || o.block_size < 32 || o.block_size > 1024 ||
        o.block_size % 32 || o.blocks_per_sm < 1 || o.pool_bytes < 0 || o.reserve_bytes < 0 ||
        o.idle_timeout_ns <= 0 || o.poll_interval_us < 0 || o.exclusive_min_edges < 0 ||
        (o.mode != BM_APFB && o.mode != BM_APSB) ||
        (o.bfs != BM_GPUBFS && o.bfs != BM_GPUBFS_WR) || (o.deterministic != 0 && o.deterministic != 1) ||
        (o.deterministic && o.bfs != BM_GPUBFS_WR))
        return BM_ERR_INVALID_ARG;
    bm_server* s = new (std::nothrow) bm_server();
    if (!s) return BM_ERR_NOMEM;
    s->opt = o;
    auto fail = [&](int32_t rc) { bm_server_destroy(s); return rc; };
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(BM_ERR_CUDA);
    }
    int per_sm = 0;
    if ((o.deterministic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve<true, true>, o.block_size, 0)
         : o.bfs == BM_GPUBFS_WR ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve<true>, o.block_size, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve<false>, o.block_size, 0)) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(BM_ERR_CUDA);
    }
    if (per_sm < 1) return fail(BM_ERR_UNSUPPORTED);
    s->block = o.block_size;
    // alongside: one worker block per SM, leaving the other half of each SM to the whole-GPU lane
    const int bps = o.exclusive_alongside ? 1 : (o.blocks_per_sm < per_sm ? o.blocks_per_sm : per_sm);
    s->grid = s->num_sms * bps;
    size_t pool = (size_t)o.pool_bytes;
    if (pool == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { (void)cudaGetLastError(); return fail(BM_ERR_CUDA); }
        pool = fr > (size_t)o.reserve_bytes ? fr - (size_t)o.reserve_bytes : 0;
    }
    if (pool < 4096) return fail(BM_ERR_NOMEM);
    if (cudaMalloc(&s->pool, pool) != cudaSuccess) { (void)cudaGetLastError(); return fail(BM_ERR_NOMEM); }
    s->alloc = new (std::nothrow) PoolAllocator(pool);
    const size_t mbytes = sizeof(MappedHead) + (sizeof(SlotDesc) + sizeof(SlotDone)) * (size_t)o.ring_slots;
    if (!s->alloc || cudaHostAlloc(&s->mapped, mbytes, cudaHostAllocMapped) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(BM_ERR_NOMEM);
    }
    memset(s->mapped, 0, mbytes);
    s->head = (MappedHead*)s->mapped;
    s->desc = (SlotDesc*)((char*)s->mapped + sizeof(MappedHead));
    s->done = (SlotDone*)((char*)s->mapped + sizeof(MappedHead) + sizeof(SlotDesc) * (size_t)o.ring_slots);
    if (cudaHostGetDevicePointer(&s->d_mapped, s->mapped, 0) != cudaSuccess ||
        cudaMalloc((void**)&s->d_claimed, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(s->d_claimed, 0, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->work_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->excl_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->worker_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_excl_ctl, sizeof(bmd::Ctl) * kExclSlots) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(BM_ERR_CUDA);
    }
    s->d_busy = (int32_t*)(s->d_claimed + 1);
    for (int k = 0; k < kExclSlots; ++k) {
        if (cudaEventCreateWithFlags(&s->excl_ev[k], cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(BM_ERR_CUDA);
        }
        s->excl_free.push_back(kExclSlots - 1 - k);
    }
    s->ring_owner.assign((size_t)o.ring_slots, -1);
    s->running = true;
    s->sched = std::thread(scheduler_main, s);
    *out = s;
    return BM_OK;
}

int32_t bm_server_submit(bm_server* s, int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* h_col_ptr,
                         const int32_t* h_row_idx, int32_t greedy, int64_t* id_out) {
    bmi::NvtxRange nvtx_range("bm_server_submit");
    if (!s || !id_out || n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL || !h_col_ptr ||
        (!h_row_idx && nnz > 0))
        return BM_ERR_INVALID_ARG;
    if (s->sticky) return BM_ERR_STATE;
    std::lock_guard<std::mutex> lk(s->mu);
    Request r;
    r.id = s->next_id++;
    r.nr = n_rows;
    r.nc = n_cols;
    r.nnz = nnz;
    r.h_cp = h_col_ptr;
    r.h_ri = h_row_idx;
    r.greedy = greedy ? 1 : 0;
    r.t_submit = std::chrono::steady_clock::now();
    s->reqs.emplace(r.id, r);
    s->pending.push_back(r.id);
    *id_out = r.id;
    return BM_OK;
}

int32_t bm_server_poll(bm_server* s, int64_t id, bm_request_info* info) {
    if (!s || !info) return BM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BM_ERR_INVALID_ARG;
    const Request& r = it->second;
    memset(info, 0, sizeof(*info));
    info->state = r.state;
    info->card = r.card;
    info->status = r.status;
    info->phases = r.phases;
    if (r.state == DONE)
        info->latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r.t_done - r.t_submit).count();
    return s->sticky ? s->sticky : BM_OK;
}

int32_t bm_server_wait(bm_server* s, int64_t id, int64_t timeout_ns, bm_request_info* info) {
    bmi::NvtxRange nvtx_range("bm_server_wait");
    if (!s || !info) return BM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BM_ERR_INVALID_ARG;
    if (timeout_ns < 0) timeout_ns = 0;
    if (timeout_ns > 3600000000000ll) timeout_ns = 3600000000000ll;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
    while (it->second.state != DONE && it->second.state != CANCELLED && !s->sticky) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) break;
        it = s->reqs.find(id);
    }
    const Request& r = it->second;
    memset(info, 0, sizeof(*info));
    info->state = r.state;
    info->card = r.card;
    info->status = r.status;
    info->phases = r.phases;
    if (r.state == DONE)
        info->latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r.t_done - r.t_submit).count();
    if (s->sticky) return s->sticky;
    return (r.state == DONE || r.state == CANCELLED) ? BM_OK : BM_ERR_TIMEOUT;
}

int32_t bm_server_cancel(bm_server* s, int64_t id) {
    if (!s) return BM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BM_ERR_INVALID_ARG;
    if (it->second.state != PENDING) return BM_ERR_STATE;  // already admitted
    it->second.state = CANCELLED;
    s->cv.notify_all();
    return BM_OK;
}

int32_t bm_server_fetch(bm_server* s, int64_t id, int32_t* h_rmatch, int32_t* h_cmatch) {
    if (!s) return BM_ERR_INVALID_ARG;
    size_t orm = 0, ocm = 0;
    int32_t nr = 0, nc = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return BM_ERR_INVALID_ARG;
        const Request& r = it->second;
        if (r.state != DONE || !r.has_mem || r.status != 0) return BM_ERR_STATE;
        orm = r.off_rm;
        ocm = r.off_cm;
        nr = r.nr;
        nc = r.nc;
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return BM_ERR_CUDA;
    if (h_rmatch && nr) cudaMemcpyAsync(h_rmatch, s->pool + orm, 4 * (size_t)nr, cudaMemcpyDeviceToHost, st);
    if (h_cmatch && nc) cudaMemcpyAsync(h_cmatch, s->pool + ocm, 4 * (size_t)nc, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return e == cudaSuccess ? BM_OK : BM_ERR_CUDA;
}

int32_t bm_server_release(bm_server* s, int64_t id) {
    if (!s) return BM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BM_ERR_INVALID_ARG;
    Request& r = it->second;
    if (r.state != DONE && r.state != CANCELLED) return BM_ERR_STATE;
    if (r.has_mem) s->alloc->release(r.off, r.bytes);
    if (r.uploaded) cudaEventDestroy(r.uploaded);
    s->reqs.erase(it);
    return BM_OK;
}

int32_t bm_server_get_stats(bm_server* s, bm_server_stats* st) {
    if (!s || !st) return BM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->pending = (int64_t)s->pending.size();
    st->inflight = s->inflight;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->worker_launches = s->launches;
    st->pool_bytes = (int64_t)s->alloc->size();
    st->pool_used = (int64_t)s->alloc->used();
    st->grid = s->grid;
    st->block = s->block;
    st->exclusive_runs = s->exclusive_runs;
    return s->sticky;
}

int32_t bm_server_destroy(bm_server* s) {
    if (!s) return BM_ERR_INVALID_ARG;
    if (s->running.load()) {
        s->running = false;
        if (s->sched.joinable()) s->sched.join();
    }
    if (s->head) __atomic_store_n(&s->head->stop, 1, __ATOMIC_RELEASE);
    if (s->work_stream) cudaStreamSynchronize(s->work_stream);
    if (s->excl_stream) cudaStreamSynchronize(s->excl_stream);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    for (auto& kv : s->reqs)
        if (kv.second.uploaded) cudaEventDestroy(kv.second.uploaded);
    if (s->worker_ev) cudaEventDestroy(s->worker_ev);
    for (int k = 0; k < kExclSlots; ++k)
        if (s->excl_ev[k]) cudaEventDestroy(s->excl_ev[k]);
    if (s->h_excl_ctl) cudaFreeHost(s->h_excl_ctl);
    if (s->work_stream) cudaStreamDestroy(s->work_stream);
    if (s->excl_stream) cudaStreamDestroy(s->excl_stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->d_claimed) cudaFree(s->d_claimed);
    if (s->mapped) cudaFreeHost(s->mapped);
    if (s->pool) cudaFree(s->pool);
    delete s->alloc;
    (void)cudaGetLastError();
    delete s;
    return BM_OK;
}

}  // extern "C"
