// Interface between the library's translation units (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "bm_device.cuh"

namespace bmi {

// NVTX range over one C-ABI call (header-only NVTX: free unless a profiler
// that reads NVTX is attached), so that timelines show which call launched
// which kernels.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Enqueues on `st`, without waiting, the whole method on one graph over the
// whole GPU (the persistent single-graph kernel):
//   the control block p.ctl cleared; the CSR checked (BM_ERR_INVALID_CSR in
//   p.ctl->err, and nothing below then reads it); rmatch / cmatch set to
//   unmatched and the claim stamps p.rvis to zero; the cheap matching if
//   `greedy`; one cooperative launch of the persistent kernel.
// p must hold the graph (n_rows/n_cols, device col_ptr/row_idx with nnz
// edges), the matching arrays and the workspace of a context's launch:
// level, root (n_cols), pred, endpoints, rvis (n_rows), queue, queue2, crec
// (n_cols), ctl; mode and one_ep select the variant (GPUBFS-WR when wr).
// The outcome (status, |M|, phases) is in p.ctl when the stream reaches it.
// Returns BM_OK, or BM_ERR_CUDA / BM_ERR_UNSUPPORTED when a launch failed.
// blocks_per_sm > 0 caps the cooperative grid at that many blocks per SM (a
// launch that shares the GPU with other resident kernels); 0 = as many as fit.
int32_t enqueue_match(bmd::Params p, long long nnz, bool wr, int greedy, cudaStream_t st, int blocks_per_sm = 0);

}  // namespace bmi
