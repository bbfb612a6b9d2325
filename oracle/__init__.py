"""Oracle for maximum cardinality bipartite matching -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package.  It shares no code with the CUDA path.

* ``bm_oracle.c`` (compiled here with the host C compiler, loaded by ctypes):
  greedy initial matching, Hopcroft-Karp, matching validation, the Koenig
  certificate, the alternating-BFS levels and the method itself run level by
  level with fixed tie-break rules -- see that file's header for the passages
  of arXiv 1303.1379 each one follows.
* pure Python, for tiny graphs only: exhaustive search over edge subsets and a
  dynamic program over row bitmasks, both straight from the definition of a
  maximum matching (Section 2).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

I32P = ctypes.POINTER(ctypes.c_int32)
I64P = ctypes.POINTER(ctypes.c_int64)
U8P = ctypes.POINTER(ctypes.c_uint8)

ERRORS = {
    0: "ok", -1: "bad argument", -2: "out of memory", -3: "match index out of range",
    -4: "rmatch and cmatch are not inverse", -5: "matched pair is not an edge",
    -6: "augmenting path exists (not maximum)", -7: "edge not covered",
    -8: "cover size differs from |M|",
}


def build(force: bool = False) -> str:
    """Compile bm_oracle.c into liboracle.so (OpenMP only for the batch helper)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fvisibility=hidden", _SRC,
            "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            g6 = [ctypes.c_int32, ctypes.c_int32, I32P, I32P, I32P, I32P]
            lib.orc_csr_check.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, I32P, I32P]
            lib.orc_csr_check.restype = ctypes.c_int
            lib.orc_greedy.argtypes = g6
            lib.orc_greedy.restype = ctypes.c_int64
            lib.orc_validate.argtypes = g6 + [I64P]
            lib.orc_validate.restype = ctypes.c_int
            lib.orc_hopcroft_karp.argtypes = g6 + [I64P]
            lib.orc_hopcroft_karp.restype = ctypes.c_int64
            lib.orc_konig.argtypes = g6 + [I64P]
            lib.orc_konig.restype = ctypes.c_int
            lib.orc_bfs_levels.argtypes = g6 + [ctypes.c_int32, I32P, U8P]
            lib.orc_bfs_levels.restype = ctypes.c_int64
            lib.orc_hk_batch.argtypes = [ctypes.c_int32, I32P, I32P, I64P, I64P, I64P, I32P, I32P,
                                         I32P, I32P, ctypes.c_int32, I64P]
            lib.orc_hk_batch.restype = ctypes.c_int
            lib.orc_greedy_rounds.argtypes = g6 + [I64P]
            lib.orc_greedy_rounds.restype = ctypes.c_int64
            lib.orc_apfb_wr_det.argtypes = g6 + [ctypes.c_int32, I64P]
            lib.orc_apfb_wr_det.restype = ctypes.c_int64
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t=I32P):
    return a.ctypes.data_as(t)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def empty_matching(n_rows: int, n_cols: int):
    return np.full(n_rows, -1, np.int32), np.full(n_cols, -1, np.int32)


def csr_check(n_rows, n_cols, col_ptr, row_idx) -> int:
    cp, ri = _i32(col_ptr), _i32(row_idx)
    return int(_load().orc_csr_check(n_rows, n_cols, int(ri.shape[0]), _p(cp), _p(ri)))


def greedy(n_rows, n_cols, col_ptr, row_idx):
    """Cheap matching: columns in order, each takes its first unmatched row."""
    cp, ri = _i32(col_ptr), _i32(row_idx)
    rm, cm = empty_matching(n_rows, n_cols)
    card = _load().orc_greedy(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm))
    return rm, cm, int(card)


def hopcroft_karp(n_rows, n_cols, col_ptr, row_idx, rmatch=None, cmatch=None):
    """Maximum matching by Hopcroft-Karp from an optional initial matching.
    Returns (rmatch, cmatch, |M|, phases)."""
    cp, ri = _i32(col_ptr), _i32(row_idx)
    if rmatch is None:
        rm, cm = empty_matching(n_rows, n_cols)
    else:
        rm, cm = _i32(rmatch).copy(), _i32(cmatch).copy()
    phases = np.zeros(1, np.int64)
    card = _load().orc_hopcroft_karp(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm),
                                     _p(phases, I64P))
    if card < 0:
        raise ValueError(f"hopcroft_karp: {ERRORS.get(int(card), card)}")
    return rm, cm, int(card), int(phases[0])


def validate(n_rows, n_cols, col_ptr, row_idx, rmatch, cmatch):
    """Returns (status, |M|): status 0 when (rmatch, cmatch) is a matching."""
    cp, ri, rm, cm = _i32(col_ptr), _i32(row_idx), _i32(rmatch), _i32(cmatch)
    card = np.zeros(1, np.int64)
    rc = _load().orc_validate(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm), _p(card, I64P))
    return int(rc), int(card[0])


def konig(n_rows, n_cols, col_ptr, row_idx, rmatch, cmatch):
    """Returns (status, cover size): status 0 proves the matching is maximum."""
    cp, ri, rm, cm = _i32(col_ptr), _i32(row_idx), _i32(rmatch), _i32(cmatch)
    cover = np.zeros(1, np.int64)
    rc = _load().orc_konig(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm), _p(cover, I64P))
    return int(rc), int(cover[0])


def bfs_levels(n_rows, n_cols, col_ptr, row_idx, rmatch, cmatch, L0=2):
    """Alternating BFS from all free columns for a fixed matching.
    Returns (level[nc], reached_free_row[nr] as bool)."""
    cp, ri, rm, cm = _i32(col_ptr), _i32(row_idx), _i32(rmatch), _i32(cmatch)
    level = np.zeros(n_cols, np.int32)
    reached = np.zeros(max(n_rows, 1), np.uint8)
    rc = _load().orc_bfs_levels(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm), L0, _p(level),
                                _p(reached, U8P))
    if rc < 0:
        raise MemoryError("bfs_levels")
    return level, reached[:n_rows].astype(bool)


def hk_batch(batch, greedy_first=True):
    """Hopcroft-Karp on every graph of a concatenated batch (see synth.Batch).
    Returns (rmatch, cmatch, card[G])."""
    lib = _load()
    G = batch.n_graphs
    rm = np.full(int(batch.row_off[-1]), -1, np.int32)
    cm = np.full(int(batch.col_off[-1]), -1, np.int32)
    card = np.zeros(G, np.int64)
    rc = lib.orc_hk_batch(G, _p(_i32(batch.n_rows)), _p(_i32(batch.n_cols)),
                          _p(batch.row_off, I64P), _p(batch.col_off, I64P),
                          _p(batch.edge_off, I64P), _p(_i32(batch.col_ptr)),
                          _p(_i32(batch.row_idx)), _p(rm), _p(cm), int(bool(greedy_first)),
                          _p(card, I64P))
    if rc != 0:
        raise ValueError("hk_batch failed")
    return rm, cm, card


def greedy_rounds(n_rows, n_cols, col_ptr, row_idx, rmatch=None, cmatch=None):
    """Cheap matching by rounds of proposals: each unmatched column proposes
    to the first unmatched row of its list, each row takes the smallest
    proposer.  Returns (rmatch, cmatch, |M|, rounds)."""
    cp, ri = _i32(col_ptr), _i32(row_idx)
    if rmatch is None:
        rm, cm = empty_matching(n_rows, n_cols)
    else:
        rm, cm = _i32(rmatch).copy(), _i32(cmatch).copy()
    card = np.zeros(1, np.int64)
    rounds = _load().orc_greedy_rounds(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm), _p(card, I64P))
    if rounds < 0:
        raise MemoryError("greedy_rounds")
    return rm, cm, int(card[0]), int(rounds)


DET_STATS = ("phases", "levels", "endpoints", "inserted", "columns_expanded", "edges_scanned",
             "edges_to_matched", "alternate_steps", "roots")


def apfb_wr_det(n_rows, n_cols, col_ptr, row_idx, rmatch=None, cmatch=None, apsb=False):
    """The method (Algorithm 1 with GPUBFS-WR, one endpoint per root, and
    Alternate) run level by level with the smallest-id tie-break rules of
    orc_apfb_wr_det, from an optional valid initial matching.
    Returns (rmatch, cmatch, |M|, stats dict keyed by DET_STATS)."""
    cp, ri = _i32(col_ptr), _i32(row_idx)
    if rmatch is None:
        rm, cm = empty_matching(n_rows, n_cols)
    else:
        rm, cm = _i32(rmatch).copy(), _i32(cmatch).copy()
    st = np.zeros(len(DET_STATS), np.int64)
    card = _load().orc_apfb_wr_det(n_rows, n_cols, _p(cp), _p(ri), _p(rm), _p(cm), int(bool(apsb)),
                                   _p(st, I64P))
    if card < 0:
        raise MemoryError("apfb_wr_det")
    return rm, cm, int(card), dict(zip(DET_STATS, (int(x) for x in st)))


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- tiny graphs
def edges_of(col_ptr, row_idx):
    out = []
    for c in range(len(col_ptr) - 1):
        for e in range(int(col_ptr[c]), int(col_ptr[c + 1])):
            out.append((int(row_idx[e]), c))
    return out


def brute_force_max_matching(edges) -> int:
    """Largest k such that some k edges share no vertex (exhaustive; tiny graphs)."""
    edges = list(edges)
    for k in range(len(edges), 0, -1):
        for sub in itertools.combinations(edges, k):
            rows = {r for r, _ in sub}
            cols = {c for _, c in sub}
            if len(rows) == k and len(cols) == k:
                return k
    return 0


def dp_max_matching(n_rows, col_ptr, row_idx) -> int:
    """Maximum matching by a DP over the set of used rows (n_rows <= 16):
    best[mask] = most columns matched so far using exactly the rows in mask."""
    assert n_rows <= 16
    NEG = -1
    best = [NEG] * (1 << n_rows)
    best[0] = 0
    for c in range(len(col_ptr) - 1):
        new = list(best)  # column c left unmatched
        for mask in range(1 << n_rows):
            if best[mask] == NEG:
                continue
            for e in range(int(col_ptr[c]), int(col_ptr[c + 1])):
                r = int(row_idx[e])
                if not (mask >> r) & 1:
                    m2 = mask | (1 << r)
                    if best[mask] + 1 > new[m2]:
                        new[m2] = best[mask] + 1
        best = new
    return max(best)
