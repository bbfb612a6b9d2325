"""Shared test helpers: move a synthetic graph to the GPU, run the CUDA path
through the C-ABI binding, and check its output against the oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1303_1379_gb300 import bmatch
from paper_1303_1379_gb300.synth import Graph

VARIANTS = [
    # (mode, bfs, wr_one_endpoint, driver)
    dict(mode=0, bfs=1, wr_one_endpoint=1, driver=0),  # APFB GPUBFS-WR (default)
    dict(mode=0, bfs=1, wr_one_endpoint=0, driver=0),  # APFB GPUBFS-WR as printed
    dict(mode=0, bfs=0, wr_one_endpoint=1, driver=0),  # APFB GPUBFS
    dict(mode=1, bfs=1, wr_one_endpoint=1, driver=0),  # APsB GPUBFS-WR (-(row) refinement)
    dict(mode=1, bfs=1, wr_one_endpoint=0, driver=0),  # APsB GPUBFS-WR as printed
    dict(mode=1, bfs=0, wr_one_endpoint=1, driver=0),  # APsB GPUBFS
    dict(mode=0, bfs=1, wr_one_endpoint=1, driver=1),  # host-driven loop
    dict(mode=1, bfs=0, wr_one_endpoint=1, driver=1),
]


def vname(v):
    return "{}-{}{}-{}".format("APsB" if v["mode"] else "APFB", "GPUBFS-WR" if v["bfs"] else "GPUBFS",
                               "" if not v["bfs"] else ("1" if v["wr_one_endpoint"] else "n"),
                               "host" if v["driver"] else "pers")


def to_dev(g: Graph):
    import torch
    cp = torch.from_numpy(np.ascontiguousarray(g.col_ptr, np.int32)).cuda()
    ri = torch.from_numpy(np.ascontiguousarray(g.row_idx, np.int32)).cuda()
    if ri.numel() == 0:
        ri = torch.zeros(1, dtype=torch.int32, device="cuda")
    return cp, ri


def gpu_match(g: Graph, init=None, **options):
    """Runs bm_match on g from `init` = (rmatch, cmatch) numpy arrays (or the
    empty matching).  Returns (rmatch, cmatch, card, stats) as numpy/ints."""
    import torch
    cp, ri = to_dev(g)
    m = bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, **options)
    try:
        if init is not None:
            m.set_matching(torch.from_numpy(init[0]).cuda(), torch.from_numpy(init[1]).cuda())
        rm = torch.empty(max(g.n_rows, 1), dtype=torch.int32, device="cuda")
        cm = torch.empty(max(g.n_cols, 1), dtype=torch.int32, device="cuda")
        res = m.match(rm, cm)
        return rm[:g.n_rows].cpu().numpy(), cm[:g.n_cols].cpu().numpy(), res.card, res.stats
    finally:
        m.close()


def assert_maximum(g: Graph, rm, cm, card, expect):
    st, c = oracle.validate(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm)
    assert st == 0, oracle.ERRORS[st]
    assert c == card == expect, (c, card, expect)
    st, cover = oracle.konig(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm)
    assert st == 0 and cover == expect, oracle.ERRORS.get(st, st)


def oracle_max(g: Graph) -> int:
    return oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2]


def csr_from_edges(n_rows, n_cols, edges, keep_order=False):
    cols = [[] for _ in range(n_cols)]
    for r, c in edges:
        cols[c].append(r)
    col_ptr = np.zeros(n_cols + 1, np.int32)
    row_idx = []
    for c in range(n_cols):
        rs = cols[c] if keep_order else sorted(set(cols[c]))
        row_idx += rs
        col_ptr[c + 1] = col_ptr[c] + len(rs)
    return Graph(n_rows, n_cols, col_ptr, np.array(row_idx, np.int32), "edges")
