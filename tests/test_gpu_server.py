"""Serving (continuous batching) against the oracle and against requests run
alone: |M| is exact whether a request runs alone or in a mix that arrives
while others are on the GPU, admission respects the memory pool, and bad or
oversized requests are reported without disturbing the others."""
import time

import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import bmatch, synth

from helpers import assert_maximum, csr_from_edges

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def mixed_requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nr = int(np.exp(rng.uniform(np.log(50), np.log(20000))))
        nc = max(1, int(round(nr * rng.uniform(0.8, 1.25))))
        mu = rng.uniform(3, 16)
        if i % 2 == 0:
            g = synth.uniform_graph(nr, nc, max(1, int(round(2 * mu - 1))), seed=1000 + i)
        else:
            n = max(nr, nc)
            scale = int(np.ceil(np.log2(max(n, 2))))
            g = synth.rmat_graph(scale, int(n * mu), seed=1000 + i, n=n)
        out.append(g)
    return out


def serving_requests(n, seed=4):
    """Request graphs of the served workload: rows log-uniform in [1,000,
    1,000,000], columns = rows x U[0.8, 1.25], mean degree U[3, 16], uniform
    and R-MAT alternating, seeded per request (the benchmark's recipe)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nr = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        nc = max(1, int(round(nr * rng.uniform(0.8, 1.25))))
        mu = rng.uniform(3, 16)
        if i % 2 == 0:
            g = synth.uniform_graph(nr, nc, max(1, int(round(2 * mu - 1))), seed=seed * 100000 + i)
        else:
            n_ = max(nr, nc)
            g = synth.rmat_graph(int(np.ceil(np.log2(n_))), int(n_ * mu), seed=seed * 100000 + i, n=n_)
        out.append(g)
    return out


@pytest.mark.slow
def test_served_full_size_requests():
    """Requests of the served workload at full size (up to a million rows
    and 16 M edges each), three copies of each of 16 graphs submitted at once,
    so that copies run concurrently with one another and with the other
    graphs.  Every result equals Hopcroft-Karp's |M|, and every matching is
    valid and carries a Koenig certificate."""
    reqs = serving_requests(16)
    want = [oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2] for g in reqs]
    with bmatch.Server(keep_results=1, pool_bytes=8 << 30) as srv:
        ids = [(k, srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)) for _ in range(3)
               for k, g in enumerate(reqs)]
        bad = []
        for j, (k, rid) in enumerate(ids):
            g = reqs[k]
            info = srv.wait(rid, timeout_s=120)
            if info["state"] != bmatch.BM_REQ_DONE or info["status"] != 0 or info["card"] != want[k]:
                bad.append((j, k, g.n_rows, g.nnz, info["state"], info["status"], info["card"], want[k]))
            else:
                rm = np.empty(g.n_rows, np.int32)
                cm = np.empty(g.n_cols, np.int32)
                srv.fetch(rid, rm, cm)
                assert_maximum(g, rm, cm, info["card"], want[k])
            srv.release(rid)
        # (submission, graph, rows, edges, state, status, |M|, expected) of every request that failed
        assert not bad, bad
        assert srv.stats()["pool_used"] == 0


def test_results_same_alone_and_in_the_mix():
    reqs = mixed_requests(40, seed=4)
    want = [oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2] for g in reqs]
    with bmatch.Server(keep_results=1, pool_bytes=1 << 30) as srv:
        # alone: one at a time
        alone = []
        for g in reqs[:10]:
            rid = srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
            info = srv.wait(rid)
            assert info["state"] == bmatch.BM_REQ_DONE and info["status"] == 0
            alone.append(info["card"])
            srv.release(rid)
        # the mix: all submitted at once, arriving while others run
        ids = [srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) for g in reqs]
        for k, (g, rid) in enumerate(zip(reqs, ids)):
            info = srv.wait(rid)
            assert info["status"] == 0 and info["card"] == want[k]
            rm = np.empty(g.n_rows, np.int32)
            cm = np.empty(g.n_cols, np.int32)
            srv.fetch(rid, rm, cm)
            assert_maximum(g, rm, cm, info["card"], want[k])
            srv.release(rid)
        assert alone == want[:10]
        st = srv.stats()
        assert st["completed"] == 50 and st["pool_used"] == 0


def test_admission_waits_for_pool_memory_and_rejects_oversized():
    reqs = mixed_requests(12, seed=9)
    need = max(4 * (g.nnz + 6 * g.n_cols + 3 * g.n_rows) for g in reqs)
    # a pool that holds only about two requests at a time
    with bmatch.Server(pool_bytes=3 * need, ring_slots=4) as srv:
        big = synth.uniform_graph(400000, 400000, 8, seed=2)  # far beyond the pool
        rid_big = srv.submit(big.n_rows, big.n_cols, big.col_ptr, big.row_idx)
        ids = [srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) for g in reqs]
        info = srv.wait(rid_big)
        assert info["status"] == bmatch.BM_ERR_TOO_LARGE
        for g, rid in zip(reqs, ids):
            info = srv.wait(rid)
            assert info["status"] == 0
            assert info["card"] == oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2]
        st = srv.stats()
        assert st["rejected"] == 1 and st["pool_used"] == 0


def test_malformed_request_and_cancel():
    good = synth.uniform_graph(3000, 3000, 5, seed=3)
    bad_ri = good.row_idx.copy()
    bad_ri[17] = 10 ** 7
    with bmatch.Server(pool_bytes=1 << 28) as srv:
        rid_bad = srv.submit(good.n_rows, good.n_cols, good.col_ptr, bad_ri)
        bad_cp = good.col_ptr.copy()
        bad_cp[5] = bad_cp[7] + 3
        rid_bad2 = srv.submit(good.n_rows, good.n_cols, bad_cp, good.row_idx)
        rid_ok = srv.submit(good.n_rows, good.n_cols, good.col_ptr, good.row_idx)
        assert srv.wait(rid_bad)["status"] == bmatch.BM_ERR_INVALID_CSR
        assert srv.wait(rid_bad2)["status"] == bmatch.BM_ERR_INVALID_CSR
        assert srv.wait(rid_ok)["card"] == oracle.hopcroft_karp(good.n_rows, good.n_cols,
                                                                good.col_ptr, good.row_idx)[2]
    # cancellation of requests that have not been admitted: a one-slot ring keeps them pending
    with bmatch.Server(pool_bytes=1 << 28, ring_slots=1) as srv:
        ids = [srv.submit(good.n_rows, good.n_cols, good.col_ptr, good.row_idx) for _ in range(6)]
        cancelled = [rid for rid in ids[2:] if srv.cancel(rid) == 0]
        for rid in ids:
            info = srv.wait(rid)
            if rid in cancelled:
                assert info["state"] == bmatch.BM_REQ_CANCELLED
            else:
                assert info["state"] == bmatch.BM_REQ_DONE and info["status"] == 0


def test_idle_workers_leave_and_come_back():
    g = synth.uniform_graph(2000, 2000, 4, seed=5)
    want = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2]
    with bmatch.Server(pool_bytes=1 << 26, idle_timeout_ns=2_000_000) as srv:
        for _ in range(3):
            rid = srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
            assert srv.wait(rid)["card"] == want
            srv.release(rid)
            time.sleep(0.05)  # longer than the idle timeout: the workers leave
        assert srv.stats()["worker_launches"] >= 2


def test_large_requests_run_alone_on_the_whole_gpu():
    """Requests with at least exclusive_min_edges edges run on the single-graph
    persistent kernel -- alone on the whole GPU, or beside the workers on one
    block per SM each (exclusive_alongside) -- while the others run on worker
    blocks; mixed in one stream, every result is exact and valid.  A malformed
    large request is reported as such and the requests behind it still run.
    With the threshold at 0 every request stays on the workers."""
    reqs = mixed_requests(24, seed=9)
    want = [oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)[2] for g in reqs]
    big = [g.nnz >= 20000 for g in reqs]
    assert any(big) and not all(big)
    bad_ri = reqs[0].row_idx.copy()
    bad_ri[len(bad_ri) // 2] = reqs[0].n_rows  # one row id out of range
    for threshold, alongside, expect_alone in ((20000, 0, sum(big) * 2), (20000, 1, sum(big) * 2), (0, 0, 0)):
        with bmatch.Server(keep_results=1, pool_bytes=1 << 30, exclusive_min_edges=threshold,
                           exclusive_alongside=alongside) as srv:
            ids = [srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) for g in reqs]
            rid_bad = srv.submit(reqs[0].n_rows, reqs[0].n_cols, reqs[0].col_ptr, bad_ri)
            ids += [srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) for g in reqs]
            for k, rid in enumerate(ids):
                g = reqs[k % len(reqs)]
                info = srv.wait(rid)
                assert info["state"] == bmatch.BM_REQ_DONE and info["status"] == 0, (k, info)
                assert info["card"] == want[k % len(reqs)]
                rm = np.empty(g.n_rows, np.int32)
                cm = np.empty(g.n_cols, np.int32)
                srv.fetch(rid, rm, cm)
                assert_maximum(g, rm, cm, info["card"], want[k % len(reqs)])
                srv.release(rid)
            assert srv.wait(rid_bad)["status"] == bmatch.BM_ERR_INVALID_CSR
            srv.release(rid_bad)
            st = srv.stats()
            assert st["exclusive_runs"] == expect_alone + (threshold > 0 and big[0])
            assert st["pool_used"] == 0
