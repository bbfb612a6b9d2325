// Batched matching: many independent graphs in one persistent launch.
//
// Each block runs the whole method (cheap matching, then Algorithm 1 of
// arXiv 1303.1379 with APFB/APsB and GPUBFS/GPUBFS-WR) on one graph at a time,
// taking graphs from an atomic counter in largest-first order (longest
// processing time first).  Inside a graph the steps are separated by
// __syncthreads only -- no block ever waits for another -- and the queue and
// endpoint counters live in shared memory.  The level expansion is the same
// tile code as the single-graph path (bm_device.cuh).  The launch is captured
// once in a CUDA graph and replayed by every bm_batch_match.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "bm_device.cuh"
#include "bm_internal.h"
#include "bmatch.h"

using bmd::Counters;
using bmd::L0;
using bmd::Params;
using bmd::Smem;

namespace {

// Device-side control block of a batch launch (cleared before every launch).
struct alignas(128) BatchCtl {
    int32_t next;        // next position in the largest-first order
    int32_t err;         // first error of any graph
    int32_t pad[30];
    long long phases, levels, cols, edges, endpoints, fixes, em, alt, ins;
};

struct BatchParams {
    int32_t n_graphs;
    int32_t greedy;
    int32_t mode, bfs_wr, one_ep;
    int32_t pad;
    const int32_t* order;  // graph ids, largest first
    const int32_t* n_rows;
    const int32_t* n_cols;
    const int64_t* row_off;
    const int64_t* col_off;
    const int64_t* edge_off;
    const int32_t* col_ptr;
    const int32_t* row_idx;
    int32_t* rmatch;
    int32_t* cmatch;
    int32_t* level;
    int32_t* root;
    int32_t* pred;
    int2* queue;
    int32_t* endpoints;
    unsigned long long* dkey;  // deterministic option: per column, per row; rows listed per level
    unsigned long long* ekey;
    int32_t* ecand;
    int32_t* card_out;    // [n_graphs]
    int32_t* status_out;  // [n_graphs]
    int32_t* phases_out;  // [n_graphs]
    BatchCtl* ctl;
};

// DET: the deterministic option (block_match_graph_det; GPUBFS-WR, one
// endpoint per root, the cheap matching in rounds).
template <bool WR, bool DET = false>
__global__ void __launch_bounds__(1024, 1) k_batch(BatchParams bp) {
    __shared__ Smem sm;
    __shared__ unsigned s_vis[bmd::SB_MAX_COLS / 32], s_srv[bmd::SB_MAX_COLS / 32];  // see block_match_graph
    Counters cnt{0, 0, 0, 0, 0};
    long long lv_all = 0, ep_all = 0, ph_all = 0, ins_all = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(&bp.ctl->next, 1);
        __syncthreads();
        const int pos = sm.tile;
        if (pos >= bp.n_graphs) break;
        const int g = bp.order[pos];
        Params p{};
        p.nr = bp.n_rows[g];
        p.nc = bp.n_cols[g];
        const long long ro = bp.row_off[g], co = bp.col_off[g], eo = bp.edge_off[g];
        p.col_ptr = bp.col_ptr + co + g;
        p.row_idx = bp.row_idx + eo;
        p.rmatch = bp.rmatch + ro;
        p.cmatch = bp.cmatch + co;
        p.level = bp.level + co;
        p.root = bp.root + co;
        p.pred = bp.pred + ro;
        p.queue = bp.queue + co;
        p.endpoints = bp.endpoints + ro;
        p.mode = bp.mode;
        p.one_ep = bp.one_ep;
        p.chk = &bp.ctl->err;
        int card = 0, phases = 0;
        long long levels = 0, eps = 0, ins = 0;
        int st;
        if constexpr (DET) {
            p.dkey = bp.dkey + co;
            p.ekey = bp.ekey + ro;
            p.ecand = bp.ecand + ro;
            if (p.nc <= bmd::SB_MAX_COLS) {  // visited marks in shared memory
                p.vis = s_vis;
                st = bmd::block_match_graph_det<true, true>(p, bp.greedy, sm, cnt, card, phases, levels, eps, ins);
            } else {
                st = bmd::block_match_graph_det<true>(p, bp.greedy, sm, cnt, card, phases, levels, eps, ins);
            }
        } else if (WR && bp.one_ep && p.nc <= bmd::SB_MAX_COLS) {  // tree marks in shared memory
            p.vis = s_vis;
            p.srv = s_srv;
            st = bmd::block_match_graph<WR, true, true, WR>(p, bp.greedy, sm, cnt, card, phases, levels, eps, ins);
        } else {
            st = bmd::block_match_graph<WR, true, true>(p, bp.greedy, sm, cnt, card, phases, levels, eps, ins);
        }
        if (threadIdx.x == 0) {
            bp.card_out[g] = card;
            bp.status_out[g] = st;
            bp.phases_out[g] = phases;
            if (st) atomicCAS(&bp.ctl->err, 0, st);
            lv_all += levels;
            ep_all += eps;
            ph_all += phases;
            ins_all += ins;
        }
        __syncthreads();  // sm.tile / sm.ok are rewritten for the next graph
    }
    // counters: one atomic per warp
    long long a = cnt.cols, b = cnt.edges, f = cnt.fixes, m = cnt.em, t2 = cnt.alt;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        a += __shfl_down_sync(bmd::FULL, a, s);
        b += __shfl_down_sync(bmd::FULL, b, s);
        f += __shfl_down_sync(bmd::FULL, f, s);
        m += __shfl_down_sync(bmd::FULL, m, s);
        t2 += __shfl_down_sync(bmd::FULL, t2, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long*)&bp.ctl->cols, (unsigned long long)a);
        atomicAdd((unsigned long long*)&bp.ctl->edges, (unsigned long long)b);
        atomicAdd((unsigned long long*)&bp.ctl->fixes, (unsigned long long)f);
        atomicAdd((unsigned long long*)&bp.ctl->em, (unsigned long long)m);
        atomicAdd((unsigned long long*)&bp.ctl->alt, (unsigned long long)t2);
    }
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long*)&bp.ctl->levels, (unsigned long long)lv_all);
        atomicAdd((unsigned long long*)&bp.ctl->endpoints, (unsigned long long)ep_all);
        atomicAdd((unsigned long long*)&bp.ctl->phases, (unsigned long long)ph_all);
        atomicAdd((unsigned long long*)&bp.ctl->ins, (unsigned long long)ins_all);
    }
}

// Validates every graph's local CSR (one block per graph at a time).
__global__ void k_batch_check(int G, const int32_t* n_rows, const int32_t* n_cols, const int64_t* row_off,
                              const int64_t* col_off, const int64_t* edge_off, const int32_t* col_ptr,
                              const int32_t* row_idx, BatchCtl* ctl) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int nr = n_rows[g], nc = n_cols[g];
        const int32_t* cp = col_ptr + col_off[g] + g;
        const int32_t* ri = row_idx + edge_off[g];
        const long long nnz = edge_off[g + 1] - edge_off[g];
        bool bad = false;
        if (threadIdx.x == 0 && (nr < 0 || nc < 0 || row_off[g + 1] - row_off[g] != nr ||
                                 col_off[g + 1] - col_off[g] != nc || cp[0] != 0 ||
                                 (long long)cp[nc] != nnz))
            bad = true;
        if (nc >= 0 && col_off[g + 1] - col_off[g] == nc) {
            for (int c = threadIdx.x; c < nc; c += blockDim.x)
                if (cp[c + 1] < cp[c]) bad = true;
            for (long long e = threadIdx.x; e < nnz; e += blockDim.x)
                if (ri[e] < 0 || ri[e] >= nr) bad = true;
        }
        if (bad) atomicCAS(&ctl->err, 0, BM_ERR_INVALID_CSR);
    }
}

}  // namespace

struct bm_batch {
    bm_batch_desc d{};
    int64_t total_rows = 0, total_cols = 0, total_edges = 0;
    cudaStream_t stream = nullptr;
    bm_options opt{};
    int block = 512, grid = 0, num_sms = 0;
    void* arena = nullptr;
    int32_t *order = nullptr, *level = nullptr, *root = nullptr, *pred = nullptr, *endpoints = nullptr,
            *card = nullptr, *status = nullptr, *phases = nullptr;
    int2* queue = nullptr;
    BatchCtl* ctl = nullptr;
    BatchCtl* h_ctl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* det_arena = nullptr;  // deterministic option, allocated on first use: [dkey cols][ekey rows][ecand rows]
    int32_t* g_rmatch = nullptr;  // matching arrays the captured launch points at
    int32_t* g_cmatch = nullptr;
    int g_greedy = -1;
    int32_t sticky = 0;
};

namespace {

int32_t batch_fail(bm_batch* b, cudaError_t e) {
    (void)cudaGetLastError();
    if (b) b->sticky = BM_ERR_CUDA;
    return e == cudaErrorMemoryAllocation ? BM_ERR_NOMEM : BM_ERR_CUDA;
}

#define BB_CUDA(b, call)                                     \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return batch_fail((b), e_);   \
    } while (0)

BatchParams batch_params(bm_batch* b, int32_t* rmatch, int32_t* cmatch, int greedy) {
    BatchParams bp{};
    bp.n_graphs = b->d.n_graphs;
    bp.greedy = greedy;
    bp.mode = b->opt.mode;
    bp.bfs_wr = b->opt.bfs == BM_GPUBFS_WR;
    bp.one_ep = b->opt.wr_one_endpoint;
    bp.order = b->order;
    bp.n_rows = b->d.n_rows;
    bp.n_cols = b->d.n_cols;
    bp.row_off = b->d.row_off;
    bp.col_off = b->d.col_off;
    bp.edge_off = b->d.edge_off;
    bp.col_ptr = b->d.col_ptr;
    bp.row_idx = b->d.row_idx;
    bp.rmatch = rmatch;
    bp.cmatch = cmatch;
    bp.level = b->level;
    bp.root = b->root;
    bp.pred = b->pred;
    bp.queue = b->queue;
    bp.endpoints = b->endpoints;
    if (b->det_arena) {
        const size_t cols = (size_t)(b->total_cols ? b->total_cols : 1), rows = (size_t)(b->total_rows ? b->total_rows : 1);
        char* a = (char*)b->det_arena;
        bp.dkey = (unsigned long long*)a;
        bp.ekey = (unsigned long long*)(a + ((8 * cols + 255) & ~size_t(255)));
        bp.ecand = (int32_t*)(a + ((8 * cols + 255) & ~size_t(255)) + ((8 * rows + 255) & ~size_t(255)));
    }
    bp.card_out = b->card;
    bp.status_out = b->status;
    bp.phases_out = b->phases;
    bp.ctl = b->ctl;
    return bp;
}

int32_t configure_batch(bm_batch* b) {
    b->block = b->opt.block_size ? b->opt.block_size : 512;
    int per_sm = 0;
    cudaError_t e = b->opt.deterministic
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<true, true>, b->block, 0)
                    : b->opt.bfs == BM_GPUBFS_WR
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<true>, b->block, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<false>, b->block, 0);
    if (e != cudaSuccess) return batch_fail(b, e);
    if (b->opt.blocks_per_sm > 0 && b->opt.blocks_per_sm < per_sm) per_sm = b->opt.blocks_per_sm;
    if (per_sm < 1) return BM_ERR_UNSUPPORTED;
    b->grid = per_sm * b->num_sms;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return BM_OK;
}

// Captures memset(ctl) + the persistent batch kernel into a CUDA graph.
int32_t capture(bm_batch* b, int32_t* rmatch, int32_t* cmatch, int greedy) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    cudaStream_t cs;
    BB_CUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    BatchParams bp = batch_params(b, rmatch, cmatch, greedy);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), cs);
        if (b->opt.deterministic) k_batch<true, true><<<b->grid, b->block, 0, cs>>>(bp);
        else if (b->opt.bfs == BM_GPUBFS_WR) k_batch<true><<<b->grid, b->block, 0, cs>>>(bp);
        else k_batch<false><<<b->grid, b->block, 0, cs>>>(bp);
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return batch_fail(b, e);
    b->g_rmatch = rmatch;
    b->g_cmatch = cmatch;
    b->g_greedy = greedy;
    return BM_OK;
}

}  // namespace

extern "C" {

int32_t bm_batch_create(const bm_batch_desc* desc, void* stream, const bm_options* opt, bm_batch** out) {
    bmi::NvtxRange nvtx_range("bm_batch_create");
    if (!out || !desc) return BM_ERR_INVALID_ARG;
    *out = nullptr;
    const int G = desc->n_graphs;
    if (G < 0 || !desc->n_rows || !desc->n_cols || !desc->row_off || !desc->col_off || !desc->edge_off ||
        !desc->col_ptr || (!desc->row_idx))
        return BM_ERR_INVALID_ARG;
    bm_options o;
    if (opt) o = *opt; else bm_default_options(&o);
    if (o.mode != BM_APFB && o.mode != BM_APSB) return BM_ERR_INVALID_ARG;
    if (o.bfs != BM_GPUBFS && o.bfs != BM_GPUBFS_WR) return BM_ERR_INVALID_ARG;
    if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 1024 || o.block_size % 32)) return BM_ERR_INVALID_ARG;
    if (o.deterministic != 0 && o.deterministic != 1) return BM_ERR_INVALID_ARG;
    if (o.deterministic && (o.bfs != BM_GPUBFS_WR || o.wr_one_endpoint != 1)) return BM_ERR_INVALID_ARG;
    bm_batch* b = new (std::nothrow) bm_batch();
    if (!b) return BM_ERR_NOMEM;
    b->d = *desc;
    b->stream = (cudaStream_t)stream;
    b->opt = o;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return BM_ERR_CUDA;
    }
    // offsets to the host: workspace sizes and the largest-first order
    std::vector<int64_t> ro(G + 1), co(G + 1), eo(G + 1);
    cudaStream_t st = b->stream;
    if (cudaMemcpyAsync(ro.data(), desc->row_off, 8 * (size_t)(G + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(co.data(), desc->col_off, 8 * (size_t)(G + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(eo.data(), desc->edge_off, 8 * (size_t)(G + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return BM_ERR_CUDA;
    }
    if (ro[0] != 0 || co[0] != 0 || eo[0] != 0) { delete b; return BM_ERR_INVALID_ARG; }
    for (int g = 0; g < G; ++g)
        if (ro[g + 1] < ro[g] || co[g + 1] < co[g] || eo[g + 1] < eo[g] || ro[g + 1] - ro[g] > 0x7fffffff ||
            co[g + 1] - co[g] > 0x7fffffff || eo[g + 1] - eo[g] > 0x7fffffff) {
            delete b;
            return BM_ERR_INVALID_ARG;
        }
    b->total_rows = ro[G];
    b->total_cols = co[G];
    b->total_edges = eo[G];
    std::vector<int32_t> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return eo[x + 1] - eo[x] > eo[y + 1] - eo[y];  // most edges first
    });
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t R = (size_t)(b->total_rows ? b->total_rows : 1), C = (size_t)(b->total_cols ? b->total_cols : 1);
    const size_t G1 = (size_t)(G ? G : 1);
    size_t off = 0;
    const size_t o_ctl = off; off += al(sizeof(BatchCtl));
    const size_t o_ord = off; off += al(4 * G1);
    const size_t o_card = off; off += al(4 * G1);
    const size_t o_stat = off; off += al(4 * G1);
    const size_t o_ph = off; off += al(4 * G1);
    const size_t o_lv = off; off += al(4 * C);
    const size_t o_rt = off; off += al(4 * C);
    const size_t o_q = off; off += al(8 * C);
    const size_t o_pd = off; off += al(4 * R);
    const size_t o_ep = off; off += al(4 * R);
    const size_t det_bytes = al(8 * C) + al(8 * R) + 4 * R;
    if (cudaMalloc(&b->arena, off) != cudaSuccess || cudaMallocHost((void**)&b->h_ctl, sizeof(BatchCtl)) != cudaSuccess ||
        (o.deterministic && cudaMalloc(&b->det_arena, det_bytes) != cudaSuccess)) {
        (void)cudaGetLastError();
        bm_batch_destroy(b);
        return BM_ERR_NOMEM;
    }
    char* a = (char*)b->arena;
    b->ctl = (BatchCtl*)(a + o_ctl);
    b->order = (int32_t*)(a + o_ord);
    b->card = (int32_t*)(a + o_card);
    b->status = (int32_t*)(a + o_stat);
    b->phases = (int32_t*)(a + o_ph);
    b->level = (int32_t*)(a + o_lv);
    b->root = (int32_t*)(a + o_rt);
    b->queue = (int2*)(a + o_q);
    b->pred = (int32_t*)(a + o_pd);
    b->endpoints = (int32_t*)(a + o_ep);
    int32_t rc = configure_batch(b);
    if (rc) { bm_batch_destroy(b); return rc; }
    if (cudaMemcpyAsync(b->order, order.data(), 4 * (size_t)G, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), st) != cudaSuccess) {
        (void)cudaGetLastError();
        bm_batch_destroy(b);
        return BM_ERR_CUDA;
    }
    if (G > 0) {
        k_batch_check<<<b->num_sms * 4, 256, 0, st>>>(G, desc->n_rows, desc->n_cols, desc->row_off, desc->col_off, desc->edge_off,
                                                     desc->col_ptr, desc->row_idx, b->ctl);
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        bm_batch_destroy(b);
        return BM_ERR_CUDA;
    }
    if (b->h_ctl->err) {
        rc = b->h_ctl->err;
        bm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return BM_OK;
}

int32_t bm_batch_set_options(bm_batch* b, const bm_options* opt) {
    if (!b || !opt) return BM_ERR_INVALID_ARG;
    if (b->sticky) return BM_ERR_STATE;
    if (opt->mode != BM_APFB && opt->mode != BM_APSB) return BM_ERR_INVALID_ARG;
    if (opt->bfs != BM_GPUBFS && opt->bfs != BM_GPUBFS_WR) return BM_ERR_INVALID_ARG;
    if (opt->block_size != 0 && (opt->block_size < 32 || opt->block_size > 1024 || opt->block_size % 32))
        return BM_ERR_INVALID_ARG;
    if (opt->deterministic != 0 && opt->deterministic != 1) return BM_ERR_INVALID_ARG;
    if (opt->deterministic && (opt->bfs != BM_GPUBFS_WR || opt->wr_one_endpoint != 1)) return BM_ERR_INVALID_ARG;
    if (opt->deterministic && !b->det_arena) {
        const size_t cols = (size_t)(b->total_cols ? b->total_cols : 1), rows = (size_t)(b->total_rows ? b->total_rows : 1);
        const size_t bytes = ((8 * cols + 255) & ~size_t(255)) + ((8 * rows + 255) & ~size_t(255)) + 4 * rows;
        if (cudaMalloc(&b->det_arena, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            b->det_arena = nullptr;
            return BM_ERR_NOMEM;
        }
    }
    b->opt = *opt;
    return configure_batch(b);
}

int32_t bm_batch_match(bm_batch* b, int32_t greedy, int32_t* rmatch, int32_t* cmatch, int32_t* card_out,
                       bm_batch_stats* stats) {
    bmi::NvtxRange nvtx_range("bm_batch_match");
    if (!b || ((!rmatch || !cmatch) && b->d.n_graphs > 0)) return BM_ERR_INVALID_ARG;
    if (b->sticky) return BM_ERR_STATE;
    cudaStream_t st = b->stream;
    const int G = b->d.n_graphs;
    if (G > 0) {
        if (!b->exec || b->g_rmatch != rmatch || b->g_cmatch != cmatch || b->g_greedy != (greedy ? 1 : 0)) {
            int32_t rc = capture(b, rmatch, cmatch, greedy ? 1 : 0);
            if (rc) return rc;
        }
        BB_CUDA(b, cudaGraphLaunch(b->exec, st));
        if (card_out) BB_CUDA(b, cudaMemcpyAsync(card_out, b->card, 4 * (size_t)G, cudaMemcpyDeviceToDevice, st));
    }
    BB_CUDA(b, cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
    BB_CUDA(b, cudaStreamSynchronize(st));
    const BatchCtl& h = *b->h_ctl;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->status = G > 0 ? h.err : 0;
        stats->phases = h.phases;
        stats->levels = h.levels;
        stats->columns_expanded = h.cols;
        stats->edges_scanned = h.edges;
        stats->endpoints = h.endpoints;
        stats->fix_repairs = h.fixes;
        stats->alternate_steps = h.alt;
        stats->edges_to_matched = h.em;
        stats->inserted = h.ins;
        stats->grid = b->grid;
        stats->block = b->block;
    }
    return G > 0 ? h.err : BM_OK;
}

int32_t bm_batch_graph_status(bm_batch* b, int32_t* status_out, int32_t* phases_out) {
    if (!b) return BM_ERR_INVALID_ARG;
    const int G = b->d.n_graphs;
    if (G == 0) return BM_OK;
    if (status_out) BB_CUDA(b, cudaMemcpyAsync(status_out, b->status, 4 * (size_t)G, cudaMemcpyDeviceToDevice, b->stream));
    if (phases_out) BB_CUDA(b, cudaMemcpyAsync(phases_out, b->phases, 4 * (size_t)G, cudaMemcpyDeviceToDevice, b->stream));
    BB_CUDA(b, cudaStreamSynchronize(b->stream));
    return BM_OK;
}

int32_t bm_batch_destroy(bm_batch* b) {
    if (!b) return BM_ERR_INVALID_ARG;
    if (b->arena) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->arena) cudaFree(b->arena);
    if (b->det_arena) cudaFree(b->det_arena);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    (void)cudaGetLastError();
    delete b;
    return BM_OK;
}

}  // extern "C"

extern "C" int32_t bm_batch_autotune(bm_batch* b, int32_t greedy, const int32_t* rmatch0, const int32_t* cmatch0,
                                     int32_t* rmatch_work, int32_t* cmatch_work, int32_t n_candidates,
                                     const int32_t* block_sizes, const int32_t* blocks_per_sm, int32_t reps,
                                     float* ms_out, int32_t* best_out) {
    bmi::NvtxRange nvtx_range("bm_batch_autotune");
    if (!b || !block_sizes || !blocks_per_sm || !best_out || n_candidates < 1 || reps < 1) return BM_ERR_INVALID_ARG;
    if (b->d.n_graphs > 0 && (!rmatch0 || !cmatch0 || !rmatch_work || !cmatch_work)) return BM_ERR_INVALID_ARG;
    if (b->sticky) return BM_ERR_STATE;
    cudaStream_t st = b->stream;
    cudaEvent_t e0, e1;
    BB_CUDA(b, cudaEventCreate(&e0));
    BB_CUDA(b, cudaEventCreate(&e1));
    const bm_options keep = b->opt;
    int best = -1;
    float best_ms = 0.f;
    int32_t rc = BM_OK;
    for (int i = 0; i < n_candidates && rc == BM_OK; ++i) {
        bm_options o = keep;
        o.block_size = block_sizes[i];
        o.blocks_per_sm = blocks_per_sm[i];
        float cand = -1.f;
        if (bm_batch_set_options(b, &o) == BM_OK) {
            for (int r = 0; r < reps && rc == BM_OK; ++r) {
                if (b->total_rows) cudaMemcpyAsync(rmatch_work, rmatch0, 4 * (size_t)b->total_rows, cudaMemcpyDeviceToDevice, st);
                if (b->total_cols) cudaMemcpyAsync(cmatch_work, cmatch0, 4 * (size_t)b->total_cols, cudaMemcpyDeviceToDevice, st);
                cudaEventRecord(e0, st);
                rc = bm_batch_match(b, greedy, rmatch_work, cmatch_work, nullptr, nullptr);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rc == BM_OK && (cand < 0.f || ms < cand)) cand = ms;
            }
        }
        if (ms_out) ms_out[i] = cand;
        if (cand >= 0.f && (best < 0 || cand < best_ms)) { best = i; best_ms = cand; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BM_OK) return rc;
    if (best < 0) { bm_batch_set_options(b, &keep); return BM_ERR_UNSUPPORTED; }
    bm_options o = keep;
    o.block_size = block_sizes[best];
    o.blocks_per_sm = blocks_per_sm[best];
    *best_out = best;
    return bm_batch_set_options(b, &o);
}
