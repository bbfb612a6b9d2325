"""The allocation-free entry point, bm_match_noalloc.

Some callers cannot call cudaMalloc: code that runs inside a memory pool owning
all device memory of the process, plugins whose host application forbids
allocation after start-up, real-time loops where an allocation could block or
fail.  bm_match_noalloc serves them by keeping its working arrays in a fixed
device array compiled into the library.  These tests compare it with the
context-based bm_match on the same inputs, on consecutive calls (the shared
scratch keeps the previous call's contents, so a second call must not be
affected by the first), and check the size limit.  This file is collected last
so that a failure here cannot hide another test's result.
"""
import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import bmatch, synth

from helpers import assert_maximum, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def with_context(g, rm0, cm0):
    """The existing entry point: bm_create + bm_set_matching + bm_match."""
    cp, ri = to_dev(g)
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri) as m:
        m.set_matching(torch.from_numpy(rm0).cuda(), torch.from_numpy(cm0).cuda())
        return m.match().card


def without_allocation(g, rm0, cm0):
    cp, ri = to_dev(g)
    rm = torch.from_numpy(rm0.copy()).cuda()
    cm = torch.from_numpy(cm0.copy()).cuda()
    torch.cuda.synchronize()
    rc, card = bmatch.bm_match_noalloc(g.n_rows, g.n_cols, g.nnz, cp, ri, rm, cm)
    return rc, card, rm.cpu().numpy(), cm.cpu().numpy()


def test_noalloc_agrees_with_bm_match_on_consecutive_calls():
    big = synth.rmat_graph(17, 1 << 21, seed=9)          # 131,072 x 131,072
    small = synth.uniform_graph(7919, 8111, 5, seed=21)   # ragged sizes
    cases = [
        (big, *oracle.empty_matching(big.n_rows, big.n_cols)),
        (small, *oracle.greedy(small.n_rows, small.n_cols, small.col_ptr, small.row_idx)[:2]),
        (big, *oracle.greedy(big.n_rows, big.n_cols, big.col_ptr, big.row_idx)[:2]),
    ]
    for g, rm0, cm0 in cases:
        want = with_context(g, rm0, cm0)
        rc, card, rm, cm = without_allocation(g, rm0, cm0)
        assert rc == bmatch.BM_OK, bmatch.status_string(rc)
        assert card == want
        assert_maximum(g, rm, cm, card, want)


def scratch_need(n_rows, n_cols):
    """Bytes of scratch a graph needs, as bmatch.h states the limit: 1024 bytes
    of control block plus levels, roots and queue over the columns (4, 4 and 8
    bytes each) and predecessors and endpoints over the rows (4 bytes each),
    each array rounded up to 256 bytes."""
    r = lambda b: (b + 255) // 256 * 256
    return 1024 + 2 * r(4 * n_cols) + r(8 * n_cols) + 2 * r(4 * n_rows)


def empty_graph_call(n_rows, n_cols):
    cp = torch.zeros(n_cols + 1, dtype=torch.int32, device="cuda")
    ri = torch.zeros(1, dtype=torch.int32, device="cuda")
    rm = torch.full((n_rows,), -1, dtype=torch.int32, device="cuda")
    cm = torch.full((n_cols,), -1, dtype=torch.int32, device="cuda")
    return bmatch.bm_match_noalloc(n_rows, n_cols, 0, cp, ri, rm, cm)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    limit = 32 << 20
    n = 4_000_000  # needs about 1024 + 4*(4n + 2n) bytes, far above 32 MiB
    assert scratch_need(n, n) > limit
    rc, _ = empty_graph_call(n, n)
    assert rc == bmatch.BM_ERR_TOO_LARGE
    assert bmatch.status_string(rc) != "unknown status"
    # the boundary: the largest square graph that fits runs, one more row and column does not
    n = 1_398_016
    assert scratch_need(n, n) <= limit < scratch_need(n + 1, n + 1)
    rc, card = empty_graph_call(n, n)
    assert rc == bmatch.BM_OK and card == 0
    rc, _ = empty_graph_call(n + 1, n + 1)
    assert rc == bmatch.BM_ERR_TOO_LARGE
    # rectangular: the rows' share and the columns' share are counted separately
    rc, _ = empty_graph_call(2 * n, n // 2)
    assert (rc == bmatch.BM_OK) == (scratch_need(2 * n, n // 2) <= limit)


def test_noalloc_rejects_invalid_matching_and_leaves_it_unchanged():
    g = synth.uniform_graph(500, 400, 4, seed=3)
    rm0, cm0 = oracle.empty_matching(g.n_rows, g.n_cols)
    rm0[3] = 7  # cmatch[7] does not point back
    rc, _, rm, cm = without_allocation(g, rm0, cm0)
    assert rc == bmatch.BM_ERR_INVALID_MATCHING
    assert np.array_equal(rm, rm0) and np.array_equal(cm, cm0)
