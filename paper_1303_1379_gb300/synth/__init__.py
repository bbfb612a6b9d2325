"""Seeded synthetic bipartite graphs (column CSR, int32) for tests and benchmarks.

This module draws inputs only: it contains none of the matching method's
arithmetic, and both the CUDA path's tests and the oracle's tests take their
graphs from here.  The generators live in ``synth.c`` (Philox-4x32-10 counter
based draws, see that file for the exact definitions); this wrapper compiles
it on first use with the host C compiler and calls it through ctypes.

Workloads (the shapes of the paper's sparse-matrix instances, Section 4):

* ``uniform_graph``  : column degree U{1..dmax}, distinct uniform rows.
* ``rmat_graph``     : R-MAT power law (a, b, c, d quadrant probabilities),
                       duplicates removed, ids >= n rejected.
* ``stencil_graph``  : 5-point stencil on a g x g grid with an exact number of
                       dropped diagonals and randomly dropped off-diagonals.
* ``batch_graphs``   : many uniform graphs with log-uniform sizes, concatenated.
* ``permute_graph``  : random row and column permutation of a graph.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libbmsynth.so")
_lock = threading.Lock()
_lib = None

I32P = ctypes.POINTER(ctypes.c_int32)
I64P = ctypes.POINTER(ctypes.c_int64)
U32P = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile synth.c into libbmsynth.so next to it (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fvisibility=hidden", _SRC,
            "-o", _LIB + ".tmp", "-lm"]
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
            lib.bms_philox4x32_10.argtypes = [U32P, U32P, U32P]
            lib.bms_philox4x32_10.restype = None
            lib.bms_uniform_degrees.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, I32P]
            lib.bms_uniform_degrees.restype = ctypes.c_int64
            lib.bms_uniform_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                             ctypes.c_int32, I32P, I32P]
            lib.bms_uniform_fill.restype = ctypes.c_int
            lib.bms_rmat.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, I32P, I32P]
            lib.bms_rmat.restype = ctypes.c_int64
            lib.bms_stencil.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, I32P, I32P]
            lib.bms_stencil.restype = ctypes.c_int64
            lib.bms_batch_params.argtypes = [ctypes.c_uint64, ctypes.c_int32] + \
                [ctypes.c_double] * 6 + [I32P, I32P, I32P]
            lib.bms_batch_params.restype = ctypes.c_int
            lib.bms_batch_degrees.argtypes = [ctypes.c_uint64, ctypes.c_int32, I32P, I32P, I32P,
                                              I64P, I32P, I64P]
            lib.bms_batch_degrees.restype = ctypes.c_int
            lib.bms_batch_fill.argtypes = [ctypes.c_uint64, ctypes.c_int32, I32P, I32P, I64P,
                                           I64P, I32P, I32P]
            lib.bms_batch_fill.restype = ctypes.c_int
            lib.bms_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, I32P]
            lib.bms_permutation.restype = ctypes.c_int
            lib.bms_num_threads.argtypes = []
            lib.bms_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray, t=I32P):
    return a.ctypes.data_as(t)


@dataclass
class Graph:
    """A bipartite graph in column CSR form: rows of column c are
    ``row_idx[col_ptr[c]:col_ptr[c+1]]``."""
    n_rows: int
    n_cols: int
    col_ptr: np.ndarray  # int32 [n_cols + 1]
    row_idx: np.ndarray  # int32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_ptr[-1]) if self.n_cols > 0 else 0


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox-4x32-10 block (exposed for the known-answer test)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().bms_philox4x32_10(_p(c, U32P), _p(k, U32P), _p(out, U32P))
    return out


def uniform_graph(n_rows: int, n_cols: int, dmax: int, seed: int, graph: int = 0) -> Graph:
    lib = _load()
    col_ptr = np.zeros(n_cols + 1, dtype=np.int32)
    nnz = lib.bms_uniform_degrees(seed, graph, n_rows, n_cols, dmax, _p(col_ptr))
    if nnz < 0:
        raise ValueError("uniform_graph: bad arguments")
    row_idx = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.bms_uniform_fill(seed, graph, n_rows, n_cols, _p(col_ptr), _p(row_idx))
    return Graph(n_rows, n_cols, col_ptr, row_idx[:nnz],
                 f"uniform nr={n_rows} nc={n_cols} deg U{{1..{dmax}}} seed={seed}")


def rmat_graph(scale: int, n_samples: int, seed: int, a=0.57, b=0.19, c=0.19, n: int | None = None) -> Graph:
    lib = _load()
    n = (1 << scale) if n is None else n
    col_ptr = np.zeros(n + 1, dtype=np.int32)
    buf = np.zeros(max(n_samples, 1), dtype=np.int32)
    nnz = lib.bms_rmat(seed, scale, n, n_samples, a, b, c, _p(col_ptr), _p(buf))
    if nnz < 0:
        raise ValueError("rmat_graph: bad arguments or out of memory")
    row_idx = buf[:nnz].copy()
    return Graph(n, n, col_ptr, row_idx,
                 f"rmat scale={scale} n={n} samples={n_samples} a={a} b={b} c={c} seed={seed}")


def stencil_graph(g: int, n_diag_drop: int, p_off: float, seed: int) -> Graph:
    lib = _load()
    n = g * g
    col_ptr = np.zeros(n + 1, dtype=np.int32)
    buf = np.zeros(5 * n, dtype=np.int32)
    nnz = lib.bms_stencil(seed, g, n_diag_drop, p_off, _p(col_ptr), _p(buf))
    if nnz < 0:
        raise ValueError("stencil_graph: bad arguments")
    return Graph(n, n, col_ptr, buf[:nnz].copy(),
                 f"stencil {g}x{g} diag_drop={n_diag_drop} p_off={p_off} seed={seed}")


@dataclass
class Batch:
    """Many graphs concatenated.  Graph k has ``n_rows[k]`` rows and
    ``n_cols[k]`` columns; its local col_ptr (``n_cols[k] + 1`` entries from 0)
    is ``col_ptr[col_off[k] + k : col_off[k + 1] + k + 1]`` and its local row
    ids are ``row_idx[edge_off[k] : edge_off[k + 1]]``."""
    n_rows: np.ndarray    # int32 [G]
    n_cols: np.ndarray    # int32 [G]
    row_off: np.ndarray   # int64 [G + 1]
    col_off: np.ndarray   # int64 [G + 1]
    edge_off: np.ndarray  # int64 [G + 1]
    col_ptr: np.ndarray   # int32 [sum(n_cols) + G]
    row_idx: np.ndarray   # int32 [sum(nnz)]

    @property
    def n_graphs(self) -> int:
        return int(self.n_rows.shape[0])

    def subset(self, idx) -> "Batch":
        """The graphs idx (in that order) as a batch of their own."""
        idx = np.asarray(idx, dtype=np.int64)
        nr, nc = self.n_rows[idx], self.n_cols[idx]
        ro = np.zeros(len(idx) + 1, np.int64)
        np.cumsum(nr, out=ro[1:])
        co = np.zeros(len(idx) + 1, np.int64)
        np.cumsum(nc, out=co[1:])
        cps, ris, eo = [], [], [0]
        for k in idx:
            g = self.graph(int(k))
            cps.append(g.col_ptr)
            ris.append(g.row_idx)
            eo.append(eo[-1] + g.nnz)
        return Batch(nr.copy(), nc.copy(), ro, co, np.array(eo, np.int64),
                     np.concatenate(cps) if cps else np.zeros(0, np.int32),
                     np.concatenate(ris) if ris else np.zeros(0, np.int32))

    def graph(self, k: int) -> Graph:
        cp = self.col_ptr[self.col_off[k] + k: self.col_off[k + 1] + k + 1]
        ri = self.row_idx[self.edge_off[k]: self.edge_off[k + 1]]
        return Graph(int(self.n_rows[k]), int(self.n_cols[k]), cp, ri, f"batch graph {k}")


def batch_graphs(n_graphs: int, seed: int, nr_lo=100.0, nr_hi=50000.0, aspect_lo=0.8,
                 aspect_hi=1.25, mu_lo=2.0, mu_hi=12.0) -> Batch:
    lib = _load()
    nr = np.zeros(n_graphs, dtype=np.int32)
    nc = np.zeros(n_graphs, dtype=np.int32)
    dmax = np.zeros(n_graphs, dtype=np.int32)
    if lib.bms_batch_params(seed, n_graphs, nr_lo, nr_hi, aspect_lo, aspect_hi, mu_lo, mu_hi,
                            _p(nr), _p(nc), _p(dmax)) != 0:
        raise ValueError("batch_graphs: bad arguments")
    col_off = np.zeros(n_graphs + 1, dtype=np.int64)
    np.cumsum(nc, out=col_off[1:])
    row_off = np.zeros(n_graphs + 1, dtype=np.int64)
    np.cumsum(nr, out=row_off[1:])
    col_ptr = np.zeros(int(col_off[-1]) + n_graphs, dtype=np.int32)
    ecount = np.zeros(n_graphs, dtype=np.int64)
    if lib.bms_batch_degrees(seed, n_graphs, _p(nr), _p(nc), _p(dmax), _p(col_off, I64P),
                             _p(col_ptr), _p(ecount, I64P)) != 0:
        raise ValueError("batch_graphs: a graph is too large")
    edge_off = np.zeros(n_graphs + 1, dtype=np.int64)
    np.cumsum(ecount, out=edge_off[1:])
    row_idx = np.zeros(max(int(edge_off[-1]), 1), dtype=np.int32)
    lib.bms_batch_fill(seed, n_graphs, _p(nr), _p(nc), _p(col_off, I64P), _p(edge_off, I64P),
                       _p(col_ptr), _p(row_idx))
    return Batch(nr, nc, row_off, col_off, edge_off, col_ptr, row_idx[: int(edge_off[-1])])


def permutation(n: int, seed: int, which: int) -> np.ndarray:
    perm = np.zeros(n, dtype=np.int32)
    _load().bms_permutation(seed, which, n, _p(perm))
    return perm


def permute_graph(g: Graph, seed: int) -> Graph:
    """Random row and column permutation (row r -> prow[r], column c -> pcol[c]),
    columns re-sorted; the structure (and the maximum matching size) is kept."""
    prow = permutation(g.n_rows, seed, 0)
    pcol = permutation(g.n_cols, seed, 1)
    deg = np.diff(g.col_ptr.astype(np.int64))
    new_deg = np.zeros(g.n_cols, dtype=np.int64)
    new_deg[pcol] = deg
    col_ptr = np.zeros(g.n_cols + 1, dtype=np.int64)
    np.cumsum(new_deg, out=col_ptr[1:])
    cols = np.repeat(pcol.astype(np.int64), deg)
    rows = prow[g.row_idx].astype(np.int64)
    order = np.lexsort((rows, cols))
    return Graph(g.n_rows, g.n_cols, col_ptr.astype(np.int32), rows[order].astype(np.int32),
                 g.name + f" permuted seed={seed}")


# The five workloads of the benchmark (sizes of the paper's instance classes;
# see the design notes for why each stands in for which matrices).
def workload(name: str) -> Graph:
    """Named workloads; a "-rcp" suffix applies the random row and column
    permutation of Section 4 (seed 5)."""
    if name.endswith("-rcp"):
        return permute_graph(workload(name[:-4]), seed=5)
    if name == "uniform10k":
        return uniform_graph(10_000, 10_000, 8, seed=0)
    if name == "rmat21":
        return rmat_graph(21, 1 << 25, seed=1)
    if name == "stencil2000":
        return stencil_graph(2000, 400_000, 0.05, seed=2)
    if name == "stencil500":  # the same recipe on a 500 x 500 mesh (profiling runs)
        return stencil_graph(500, 25_000, 0.05, seed=2)
    raise KeyError(name)


def num_threads() -> int:
    return int(_load().bms_num_threads())
