"""Thin ctypes binding of the C-ABI declared in include/bmatch.h.

Argument marshalling only: every step of the matching runs in libbmatch.so's
CUDA kernels.  Device buffers are passed as torch CUDA tensors (int32,
contiguous) or raw integer addresses; the stream defaults to torch's current
stream.  If the library cannot be loaded, every call raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

from . import build as _build

BM_OK = 0
BM_INCOMPLETE = 1
BM_ERR_INVALID_ARG = -1
BM_ERR_INVALID_CSR = -2
BM_ERR_NOMEM = -3
BM_ERR_ITER_LIMIT = -4
BM_ERR_TIMEOUT = -5
BM_ERR_CUDA = -6
BM_ERR_STATE = -7
BM_ERR_UNSUPPORTED = -8
BM_ERR_INVALID_MATCHING = -9
BM_ERR_TOO_LARGE = -10
BM_ERR_CHECK = -11

BM_APFB, BM_APSB = 0, 1
BM_GPUBFS, BM_GPUBFS_WR = 0, 1
BM_DRIVER_PERSISTENT, BM_DRIVER_HOST = 0, 1

class bm_server_options(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_int64), ("reserve_bytes", ctypes.c_int64),
                ("ring_slots", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("bfs", ctypes.c_int32), ("keep_results", ctypes.c_int32),
                ("idle_timeout_ns", ctypes.c_int64), ("poll_interval_us", ctypes.c_int32),
                ("exclusive_alongside", ctypes.c_int32), ("exclusive_min_edges", ctypes.c_int64),
                ("deterministic", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 2)]


class bm_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("card", ctypes.c_int32),
                ("phases", ctypes.c_int32), ("latency_ns", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 2)]


class bm_server_stats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("inflight", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("worker_launches", ctypes.c_int64), ("pool_bytes", ctypes.c_int64),
                ("pool_used", ctypes.c_int64), ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("exclusive_runs", ctypes.c_int64), ("reserved", ctypes.c_int64 * 1)]


BM_REQ_PENDING, BM_REQ_UPLOADING, BM_REQ_RUNNING, BM_REQ_DONE, BM_REQ_CANCELLED = range(5)


class bm_batch_desc(ctypes.Structure):
    _fields_ = [("n_graphs", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("n_rows", ctypes.c_void_p), ("n_cols", ctypes.c_void_p),
                ("row_off", ctypes.c_void_p), ("col_off", ctypes.c_void_p),
                ("edge_off", ctypes.c_void_p), ("col_ptr", ctypes.c_void_p),
                ("row_idx", ctypes.c_void_p)]


class bm_batch_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("phases", ctypes.c_int64),
                ("levels", ctypes.c_int64), ("columns_expanded", ctypes.c_int64),
                ("edges_scanned", ctypes.c_int64), ("endpoints", ctypes.c_int64),
                ("fix_repairs", ctypes.c_int64), ("alternate_steps", ctypes.c_int64),
                ("edges_to_matched", ctypes.c_int64), ("inserted", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 2)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


EXPORTS = ("bm_default_options", "bm_version", "bm_status_string", "bm_create", "bm_upload_csr",
           "bm_set_options", "bm_greedy", "bm_set_matching", "bm_get_matching", "bm_match",
           "bm_match_host", "bm_match_from", "bm_bfs", "bm_phase_profile", "bm_destroy", "bm_batch_create",
           "bm_batch_set_options", "bm_batch_match", "bm_batch_graph_status", "bm_batch_autotune",
           "bm_batch_destroy", "bm_match_noalloc", "bm_server_default_options", "bm_server_create",
           "bm_server_submit", "bm_server_poll", "bm_server_wait", "bm_server_cancel",
           "bm_server_fetch", "bm_server_release", "bm_server_get_stats", "bm_server_destroy")


class bm_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("bfs", ctypes.c_int32), ("driver", ctypes.c_int32),
                ("wr_one_endpoint", ctypes.c_int32), ("max_phases", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("wait_timeout_ns", ctypes.c_int64),
                ("total_timeout_ns", ctypes.c_int64), ("reserved", ctypes.c_int64 * 6)]


class bm_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("phases", ctypes.c_int32),
                ("initial_card", ctypes.c_int32), ("final_card", ctypes.c_int32),
                ("levels", ctypes.c_int64), ("max_levels_in_phase", ctypes.c_int64),
                ("columns_expanded", ctypes.c_int64), ("edges_scanned", ctypes.c_int64),
                ("endpoints", ctypes.c_int64), ("fix_repairs", ctypes.c_int64),
                ("inserted", ctypes.c_int64), ("edges_to_matched", ctypes.c_int64),
                ("alternate_steps", ctypes.c_int64), ("kernel_ns", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("roots", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lock = threading.Lock()
_lib = None
VP = ctypes.c_void_p
I32P = ctypes.POINTER(ctypes.c_int32)


def library_path() -> str:
    """libbmatch.so, or its range-checked twin libbmatch_checked.so when the
    environment sets BMATCH_CHECKED=1 (every index the kernels compute from
    data is checked; a violation returns BM_ERR_CHECK).  Read once, at the
    first load in the process."""
    return _build.LIB_CHECKED if os.environ.get("BMATCH_CHECKED") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Loads the library (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing and _build.is_stale(path):
                _build.build(checked=path == _build.LIB_CHECKED)
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
            lib = ctypes.CDLL(path)
            lib.bm_default_options.argtypes = [ctypes.POINTER(bm_options)]
            lib.bm_default_options.restype = None
            lib.bm_version.argtypes = []
            lib.bm_version.restype = ctypes.c_int32
            lib.bm_status_string.argtypes = [ctypes.c_int32]
            lib.bm_status_string.restype = ctypes.c_char_p
            lib.bm_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, VP, VP, VP,
                                      ctypes.POINTER(bm_options), ctypes.POINTER(VP)]
            lib.bm_create.restype = ctypes.c_int32
            lib.bm_upload_csr.argtypes = [VP, VP, VP]
            lib.bm_upload_csr.restype = ctypes.c_int32
            lib.bm_set_options.argtypes = [VP, ctypes.POINTER(bm_options)]
            lib.bm_set_options.restype = ctypes.c_int32
            lib.bm_greedy.argtypes = [VP, I32P]
            lib.bm_greedy.restype = ctypes.c_int32
            lib.bm_set_matching.argtypes = [VP, VP, VP]
            lib.bm_set_matching.restype = ctypes.c_int32
            lib.bm_get_matching.argtypes = [VP, VP, VP]
            lib.bm_get_matching.restype = ctypes.c_int32
            lib.bm_match.argtypes = [VP, VP, VP, I32P, ctypes.POINTER(bm_stats)]
            lib.bm_match.restype = ctypes.c_int32
            lib.bm_match_host.argtypes = [VP, VP, VP, VP, VP, I32P, ctypes.POINTER(bm_stats)]
            lib.bm_match_host.restype = ctypes.c_int32
            lib.bm_match_from.argtypes = [VP, VP, VP, VP, VP, I32P, ctypes.POINTER(bm_stats)]
            lib.bm_match_from.restype = ctypes.c_int32
            lib.bm_bfs.argtypes = [VP, VP, VP, VP, VP, I32P]
            lib.bm_bfs.restype = ctypes.c_int32
            lib.bm_phase_profile.argtypes = [VP, ctypes.c_int32, I32P, I32P, I32P, I32P, I32P]
            lib.bm_phase_profile.restype = ctypes.c_int32
            lib.bm_batch_create.argtypes = [ctypes.POINTER(bm_batch_desc), VP,
                                            ctypes.POINTER(bm_options), ctypes.POINTER(VP)]
            lib.bm_batch_create.restype = ctypes.c_int32
            lib.bm_batch_set_options.argtypes = [VP, ctypes.POINTER(bm_options)]
            lib.bm_batch_set_options.restype = ctypes.c_int32
            lib.bm_batch_match.argtypes = [VP, ctypes.c_int32, VP, VP, VP,
                                           ctypes.POINTER(bm_batch_stats)]
            lib.bm_batch_match.restype = ctypes.c_int32
            lib.bm_batch_graph_status.argtypes = [VP, VP, VP]
            lib.bm_batch_graph_status.restype = ctypes.c_int32
            lib.bm_batch_autotune.argtypes = [VP, ctypes.c_int32, VP, VP, VP, VP, ctypes.c_int32,
                                              I32P, I32P, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_float), I32P]
            lib.bm_batch_autotune.restype = ctypes.c_int32
            lib.bm_batch_destroy.argtypes = [VP]
            lib.bm_batch_destroy.restype = ctypes.c_int32
            lib.bm_server_default_options.argtypes = [ctypes.POINTER(bm_server_options)]
            lib.bm_server_default_options.restype = None
            lib.bm_server_create.argtypes = [ctypes.POINTER(bm_server_options), ctypes.POINTER(VP)]
            lib.bm_server_create.restype = ctypes.c_int32
            lib.bm_server_submit.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, VP,
                                             VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
            lib.bm_server_submit.restype = ctypes.c_int32
            lib.bm_server_poll.argtypes = [VP, ctypes.c_int64, ctypes.POINTER(bm_request_info)]
            lib.bm_server_poll.restype = ctypes.c_int32
            lib.bm_server_wait.argtypes = [VP, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.POINTER(bm_request_info)]
            lib.bm_server_wait.restype = ctypes.c_int32
            lib.bm_server_cancel.argtypes = [VP, ctypes.c_int64]
            lib.bm_server_cancel.restype = ctypes.c_int32
            lib.bm_server_fetch.argtypes = [VP, ctypes.c_int64, VP, VP]
            lib.bm_server_fetch.restype = ctypes.c_int32
            lib.bm_server_release.argtypes = [VP, ctypes.c_int64]
            lib.bm_server_release.restype = ctypes.c_int32
            lib.bm_server_get_stats.argtypes = [VP, ctypes.POINTER(bm_server_stats)]
            lib.bm_server_get_stats.restype = ctypes.c_int32
            lib.bm_server_destroy.argtypes = [VP]
            lib.bm_server_destroy.restype = ctypes.c_int32
            lib.bm_destroy.argtypes = [VP]
            lib.bm_destroy.restype = ctypes.c_int32
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().bm_status_string(int(status)).decode()


def _ptr(x) -> int | None:
    """Device address of a torch tensor (int32, contiguous), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch tensor, an address or None")
    if x.dtype != torch.int32 or not x.is_contiguous():
        raise TypeError("buffers must be contiguous int32 tensors")
    return x.data_ptr()


def _host_ptr(x) -> int | None:
    if x is None:
        return None
    import numpy as np
    if isinstance(x, np.ndarray):
        if x.dtype != np.int32 or not x.flags.c_contiguous:
            raise TypeError("host buffers must be contiguous int32 arrays")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.device.type != "cpu" or x.dtype != torch.int32 or not x.is_contiguous():
            raise TypeError("host tensors must be contiguous int32 CPU tensors")
        return x.data_ptr()
    raise TypeError("expected a numpy array or a CPU tensor")


def default_options(**kw) -> bm_options:
    o = bm_options()
    load().bm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(rc: int, what: str, allow=(BM_OK,)) -> int:
    if rc not in allow:
        raise BMError(rc, what)
    return rc


@dataclass
class MatchResult:
    status: int
    card: int
    stats: dict


class Matcher:
    """One bm_ctx.  Either borrows device CSR tensors (col_ptr, row_idx) or,
    when they are None, owns device storage for a CSR of the given sizes."""

    def __init__(self, n_rows: int, n_cols: int, nnz: int, col_ptr=None, row_idx=None,
                 stream: int | None = None, **options):
        self._lib = load()
        self.n_rows, self.n_cols, self.nnz = int(n_rows), int(n_cols), int(nnz)
        self._keep = (col_ptr, row_idx)  # keep borrowed tensors alive
        self.stream = _current_stream() if stream is None else stream
        self.options = default_options(**options)
        h = VP()
        rc = self._lib.bm_create(self.n_rows, self.n_cols, self.nnz, _ptr(col_ptr), _ptr(row_idx),
                                 self.stream, ctypes.byref(self.options), ctypes.byref(h))
        _check(rc, "bm_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **options):
        o = default_options(**{**{k: getattr(self.options, k) for k, _ in bm_options._fields_
                                  if k not in ("reserved",)}, **options})
        _check(self._lib.bm_set_options(self._h, ctypes.byref(o)), "bm_set_options")
        self.options = o

    def upload_csr(self, h_col_ptr, h_row_idx):
        _check(self._lib.bm_upload_csr(self._h, _host_ptr(h_col_ptr), _host_ptr(h_row_idx)),
               "bm_upload_csr")

    def greedy(self) -> int:
        card = ctypes.c_int32(0)
        _check(self._lib.bm_greedy(self._h, ctypes.byref(card)), "bm_greedy")
        return card.value

    def set_matching(self, rmatch=None, cmatch=None):
        _check(self._lib.bm_set_matching(self._h, _ptr(rmatch), _ptr(cmatch)), "bm_set_matching")

    def get_matching(self, rmatch_out=None, cmatch_out=None):
        _check(self._lib.bm_get_matching(self._h, _ptr(rmatch_out), _ptr(cmatch_out)),
               "bm_get_matching")

    def match(self, rmatch_out=None, cmatch_out=None, allow_incomplete=False) -> MatchResult:
        card = ctypes.c_int32(0)
        st = bm_stats()
        rc = self._lib.bm_match(self._h, _ptr(rmatch_out), _ptr(cmatch_out), ctypes.byref(card),
                                ctypes.byref(st))
        _check(rc, "bm_match", (BM_OK, BM_INCOMPLETE) if allow_incomplete else (BM_OK,))
        return MatchResult(rc, card.value, st.as_dict())

    def match_from(self, rmatch0, cmatch0, rmatch_out=None, cmatch_out=None) -> MatchResult:
        """bm_match_from: install (rmatch0, cmatch0) and match, one host sync."""
        card = ctypes.c_int32(0)
        st = bm_stats()
        rc = self._lib.bm_match_from(self._h, _ptr(rmatch0), _ptr(cmatch0), _ptr(rmatch_out),
                                     _ptr(cmatch_out), ctypes.byref(card), ctypes.byref(st))
        _check(rc, "bm_match_from")
        return MatchResult(rc, card.value, st.as_dict())

    def match_host(self, h_col_ptr, h_row_idx, h_rmatch=None, h_cmatch=None) -> MatchResult:
        card = ctypes.c_int32(0)
        st = bm_stats()
        rc = self._lib.bm_match_host(self._h, _host_ptr(h_col_ptr), _host_ptr(h_row_idx),
                                     _host_ptr(h_rmatch), _host_ptr(h_cmatch), ctypes.byref(card),
                                     ctypes.byref(st))
        _check(rc, "bm_match_host")
        return MatchResult(rc, card.value, st.as_dict())

    def phase_profile(self, cap: int = 4096):
        """Per-phase (levels, endpoints, first_ep_level, last_ep_level) of the
        last match (Fig. 2 of the paper: BFS levels per outer iteration)."""
        import numpy as np
        arrs = [np.zeros(max(cap, 1), np.int32) for _ in range(4)]
        n = ctypes.c_int32(0)
        ptrs = [a.ctypes.data_as(I32P) for a in arrs]
        _check(self._lib.bm_phase_profile(self._h, cap, *ptrs, ctypes.byref(n)), "bm_phase_profile")
        return [a[:n.value] for a in arrs]

    def bfs(self, level_out=None, root_out=None, pred_out=None, endpoints_out=None) -> int:
        n = ctypes.c_int32(0)
        _check(self._lib.bm_bfs(self._h, _ptr(level_out), _ptr(root_out), _ptr(pred_out),
                                _ptr(endpoints_out), ctypes.byref(n)), "bm_bfs")
        return n.value


def bm_match_noalloc(n_rows: int, n_cols: int, nnz: int, col_ptr, row_idx, rmatch, cmatch,
                     stream: int | None = None):
    """Allocation-free matching through the C-ABI (see bm_match_noalloc in
    bmatch.h): for callers that cannot allocate device memory.  rmatch/cmatch
    (device int32) hold the initial matching and receive the maximum one.
    Returns (status, |M|); the status is not raised so callers can see
    BM_ERR_TOO_LARGE and friends."""
    lib = load()
    fn = lib.bm_match_noalloc
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, VP, VP, VP, VP, VP, I32P]
    fn.restype = ctypes.c_int32
    card = ctypes.c_int32(0)
    st = _current_stream() if stream is None else stream
    rc = fn(int(n_rows), int(n_cols), int(nnz), _ptr(col_ptr), _ptr(row_idx), _ptr(rmatch),
            _ptr(cmatch), st, ctypes.byref(card))
    return int(rc), card.value


class Batch:
    """One bm_batch: many graphs (see synth.Batch for the layout) matched by
    one persistent launch.  The device copies of the descriptor arrays are
    kept alive by this object."""

    def __init__(self, n_rows, n_cols, row_off, col_off, edge_off, col_ptr, row_idx,
                 stream: int | None = None, **options):
        import torch
        self._lib = load()
        dev = torch.device("cuda", torch.cuda.current_device())

        def d(x, dt):
            return torch.as_tensor(x, dtype=dt).to(dev).contiguous()
        self.n_rows = d(n_rows, torch.int32)
        self.n_cols = d(n_cols, torch.int32)
        self.row_off = d(row_off, torch.int64)
        self.col_off = d(col_off, torch.int64)
        self.edge_off = d(edge_off, torch.int64)
        self.col_ptr = d(col_ptr, torch.int32)
        self.row_idx = d(row_idx, torch.int32) if len(row_idx) else torch.zeros(1, dtype=torch.int32, device=dev)
        self.n_graphs = int(self.n_rows.numel())
        self.total_rows = int(row_off[-1])
        self.total_cols = int(col_off[-1])
        self.stream = _current_stream() if stream is None else stream
        self.options = default_options(**options)
        self.desc = bm_batch_desc(self.n_graphs, 0, self.n_rows.data_ptr(), self.n_cols.data_ptr(),
                                  self.row_off.data_ptr(), self.col_off.data_ptr(),
                                  self.edge_off.data_ptr(), self.col_ptr.data_ptr(),
                                  self.row_idx.data_ptr())
        h = VP()
        _check(self._lib.bm_batch_create(ctypes.byref(self.desc), self.stream,
                                         ctypes.byref(self.options), ctypes.byref(h)),
               "bm_batch_create")
        self._h = h

    @classmethod
    def from_synth(cls, b, **options):
        return cls(b.n_rows, b.n_cols, b.row_off, b.col_off, b.edge_off, b.col_ptr, b.row_idx,
                   **options)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **options):
        o = default_options(**{**{k: getattr(self.options, k) for k, _ in bm_options._fields_
                                  if k != "reserved"}, **options})
        _check(self._lib.bm_batch_set_options(self._h, ctypes.byref(o)), "bm_batch_set_options")
        self.options = o

    def match(self, rmatch, cmatch, greedy: bool = True, card_out=None):
        """rmatch/cmatch: device int32 over the batch (initial -> maximum).
        Returns (status, stats dict)."""
        st = bm_batch_stats()
        rc = self._lib.bm_batch_match(self._h, int(bool(greedy)), _ptr(rmatch), _ptr(cmatch),
                                      _ptr(card_out), ctypes.byref(st))
        _check(rc, "bm_batch_match")
        return rc, st.as_dict()

    def graph_status(self):
        import torch
        s = torch.empty(max(self.n_graphs, 1), dtype=torch.int32, device="cuda")
        p = torch.empty(max(self.n_graphs, 1), dtype=torch.int32, device="cuda")
        _check(self._lib.bm_batch_graph_status(self._h, _ptr(s), _ptr(p)), "bm_batch_graph_status")
        return s[:self.n_graphs].cpu().numpy(), p[:self.n_graphs].cpu().numpy()

    def autotune(self, rmatch0, cmatch0, rmatch_work, cmatch_work, candidates, greedy=True, reps=2):
        """Times each (block_size, blocks_per_sm) candidate and keeps the
        fastest.  Returns (best index, [ms per candidate])."""
        n = len(candidates)
        blocks = (ctypes.c_int32 * n)(*[c[0] for c in candidates])
        bps = (ctypes.c_int32 * n)(*[c[1] for c in candidates])
        ms = (ctypes.c_float * n)()
        best = ctypes.c_int32(-1)
        _check(self._lib.bm_batch_autotune(self._h, int(bool(greedy)), _ptr(rmatch0), _ptr(cmatch0),
                                           _ptr(rmatch_work), _ptr(cmatch_work), n, blocks, bps,
                                           reps, ms, ctypes.byref(best)), "bm_batch_autotune")
        self.options.block_size, self.options.blocks_per_sm = candidates[best.value]
        return best.value, list(ms)


class Server:
    """Continuous-batching matching server (bm_server_*).  Requests are host
    CSR arrays (numpy int32 or pinned CPU tensors) kept alive by this object
    until they are released."""

    def __init__(self, **options):
        self._lib = load()
        o = bm_server_options()
        self._lib.bm_server_default_options(ctypes.byref(o))
        for k, v in options.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        self.options = o
        h = VP()
        _check(self._lib.bm_server_create(ctypes.byref(o), ctypes.byref(h)), "bm_server_create")
        self._h = h
        self._keep = {}

    def submit(self, n_rows, n_cols, col_ptr, row_idx, greedy=True) -> int:
        rid = ctypes.c_int64(0)
        nnz = int(col_ptr[-1]) if n_cols > 0 else 0
        _check(self._lib.bm_server_submit(self._h, int(n_rows), int(n_cols), nnz, _host_ptr(col_ptr),
                                          _host_ptr(row_idx) if nnz else None, int(bool(greedy)),
                                          ctypes.byref(rid)), "bm_server_submit")
        self._keep[rid.value] = (col_ptr, row_idx)
        return rid.value

    def poll(self, rid) -> dict:
        info = bm_request_info()
        _check(self._lib.bm_server_poll(self._h, int(rid), ctypes.byref(info)), "bm_server_poll")
        return {k: getattr(info, k) for k, _ in info._fields_ if k != "reserved"}

    def wait(self, rid, timeout_s=60.0) -> dict:
        info = bm_request_info()
        rc = self._lib.bm_server_wait(self._h, int(rid), int(timeout_s * 1e9), ctypes.byref(info))
        _check(rc, "bm_server_wait")
        return {k: getattr(info, k) for k, _ in info._fields_ if k != "reserved"}

    def cancel(self, rid):
        return int(self._lib.bm_server_cancel(self._h, int(rid)))

    def fetch(self, rid, rmatch, cmatch):
        _check(self._lib.bm_server_fetch(self._h, int(rid), _host_ptr(rmatch), _host_ptr(cmatch)),
               "bm_server_fetch")

    def release(self, rid):
        _check(self._lib.bm_server_release(self._h, int(rid)), "bm_server_release")
        self._keep.pop(int(rid), None)

    def stats(self) -> dict:
        st = bm_server_stats()
        _check(self._lib.bm_server_get_stats(self._h, ctypes.byref(st)), "bm_server_get_stats")
        return {k: getattr(st, k) for k, _ in st._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bm_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
