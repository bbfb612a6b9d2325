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


def test_noalloc_rejects_graphs_beyond_its_scratch():
    n = 4_000_000  # needs 4*(3n + 2n) bytes > 32 MiB
    cp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ri = torch.zeros(1, dtype=torch.int32, device="cuda")
    rm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rc, _ = bmatch.bm_match_noalloc(n, n, 0, cp, ri, rm, cm)
    assert rc == bmatch.BM_ERR_TOO_LARGE
    assert bmatch.status_string(rc) != "unknown status"


def test_noalloc_rejects_invalid_matching_and_leaves_it_unchanged():
    g = synth.uniform_graph(500, 400, 4, seed=3)
    rm0, cm0 = oracle.empty_matching(g.n_rows, g.n_cols)
    rm0[3] = 7  # cmatch[7] does not point back
    rc, _, rm, cm = without_allocation(g, rm0, cm0)
    assert rc == bmatch.BM_ERR_INVALID_MATCHING
    assert np.array_equal(rm, rm0) and np.array_equal(cm, cm0)
