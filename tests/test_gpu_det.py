"""The deterministic option on the GPU: element-by-element parity with the
oracle's level-by-level run of the method under the same smallest-id rules
(orc_apfb_wr_det), and the same result for every run and launch geometry.

With the option on, every choice the parallel search leaves to a race is a
minimum over a set that one BFS level fixes, so the CUDA path must return
exactly the oracle's rmatch and cmatch -- not just its |M| -- and exactly its
counters (phases, levels, endpoints, inserted and expanded columns, scanned
edges, Alternate steps, roots).
"""
import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import synth

from helpers import assert_maximum, gpu_match, oracle_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATS = oracle.DET_STATS

GRAPHS = {
    "uniform-ragged": lambda: synth.uniform_graph(20_011, 19_993, 6, seed=11),
    "uniform-tall": lambda: synth.uniform_graph(40_000, 9_001, 3, seed=12),
    "uniform-wide": lambda: synth.uniform_graph(9_001, 40_000, 3, seed=13),
    "rmat15": lambda: synth.rmat_graph(15, 1 << 19, seed=3),
    "rmat17-rcp": lambda: synth.permute_graph(synth.rmat_graph(17, 1 << 21, seed=4), seed=5),
    "stencil150": lambda: synth.stencil_graph(150, 2_250, 0.05, seed=2),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def start(g, how):
    if how == "empty":
        return None
    rm, cm, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    return rm, cm


def check_same_as_oracle(g, init, apsb, **options):
    rm0, cm0 = (None, None) if init is None else init
    w_rm, w_cm, w_card, w_st = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0,
                                                  apsb=apsb)
    rm, cm, card, st = gpu_match(g, init, deterministic=1, mode=1 if apsb else 0, **options)
    assert card == w_card
    assert {k: st[k] for k in STATS} == w_st
    np.testing.assert_array_equal(rm, w_rm)
    np.testing.assert_array_equal(cm, w_cm)
    return rm, cm, card, st


@pytest.mark.parametrize("apsb", [False, True], ids=["APFB", "APsB"])
@pytest.mark.parametrize("how", ["empty", "greedy"])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_same_matching_and_counters_as_the_oracle(name, how, apsb):
    g = graph(name)
    rm, cm, card, _ = check_same_as_oracle(g, start(g, how), apsb)
    assert_maximum(g, rm, cm, card, oracle_max(g))


@pytest.mark.parametrize("block", [64, 128, 256, 1024])
def test_every_block_size_gives_the_same_result(block):
    # tiles, guided ranges and the number of blocks all change with the block
    # size; the result must not
    g = graph("rmat17-rcp")
    check_same_as_oracle(g, start(g, "greedy"), False, block_size=block)
    check_same_as_oracle(g, start(g, "greedy"), False, block_size=block, blocks_per_sm=1)


def test_repeated_runs_on_one_context_agree():
    from paper_1303_1379_gb300 import bmatch
    from helpers import to_dev
    g = graph("stencil150")
    rm0, cm0 = start(g, "greedy")
    cp, ri = to_dev(g)
    m = bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, deterministic=1)
    try:
        outs = []
        for _ in range(4):
            m.set_matching(torch.from_numpy(rm0).cuda(), torch.from_numpy(cm0).cuda())
            rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
            cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
            res = m.match(rm, cm)
            outs.append((rm.cpu().numpy(), cm.cpu().numpy(), {k: res.stats[k] for k in STATS}))
        for o in outs[1:]:
            np.testing.assert_array_equal(o[0], outs[0][0])
            np.testing.assert_array_equal(o[1], outs[0][1])
            assert o[2] == outs[0][2]
        # switching the option off and on again on the same context
        m.set_options(deterministic=0)
        m.set_matching(torch.from_numpy(rm0).cuda(), torch.from_numpy(cm0).cuda())
        assert m.match().card == int((outs[0][1] >= 0).sum())
        m.set_options(deterministic=1)
        m.set_matching(torch.from_numpy(rm0).cuda(), torch.from_numpy(cm0).cuda())
        rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        m.match(rm)
        np.testing.assert_array_equal(rm.cpu().numpy(), outs[0][0])
    finally:
        m.close()


def test_degenerate_graphs():
    # no edges; one column; a column without rows among others; all matched already
    cases = [
        synth.Graph(5, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), "no edges"),
        synth.Graph(3, 1, np.array([0, 3], np.int32), np.array([0, 1, 2], np.int32), "one column"),
        synth.Graph(2, 3, np.array([0, 1, 1, 2], np.int32), np.array([1, 1], np.int32), "empty column"),
    ]
    for g in cases:
        rm, cm, card, _ = check_same_as_oracle(g, None, False)
        assert_maximum(g, rm, cm, card, oracle_max(g))
    g = graph("uniform-ragged")
    rm_max, cm_max, _, _ = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    check_same_as_oracle(g, (rm_max, cm_max), False)  # maximum already: one empty search


@pytest.mark.parametrize("name", ["rmat21", "stencil2000"])
def test_full_size_workloads_same_as_the_oracle(name):
    # the benchmark's graphs at full size, from the oracle's greedy start
    g = synth.workload(name)
    check_same_as_oracle(g, start(g, "greedy"), False)


# ------------------------------------------------------------ batched path
def oracle_batch_det(b, greedy):
    """Per graph: the cheap matching in rounds (if greedy), then the method
    with the same rules; returns the concatenated arrays and summed counters."""
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    rm_all = np.full(R, -1, np.int32)
    cm_all = np.full(C, -1, np.int32)
    tot = dict.fromkeys(STATS, 0)
    for k in range(b.n_graphs):
        g = b.graph(k)
        rm0 = cm0 = None
        if greedy:
            rm0, cm0, _, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        rm, cm, _, st = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0)
        rm_all[b.row_off[k]:b.row_off[k + 1]] = rm
        cm_all[b.col_off[k]:b.col_off[k + 1]] = cm
        for key in STATS:
            tot[key] += st[key]
    return rm_all, cm_all, tot


def run_batch_det(b, greedy, **options):
    from paper_1303_1379_gb300 import bmatch
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    rm = torch.full((max(R, 1),), -1, dtype=torch.int32, device="cuda")
    cm = torch.full((max(C, 1),), -1, dtype=torch.int32, device="cuda")
    with bmatch.Batch.from_synth(b, deterministic=1, **options) as bb:
        rc, st = bb.match(rm, cm, greedy=greedy)
        status, _ = bb.graph_status()
    assert rc == 0 and np.all(status == 0)
    return rm[:R].cpu().numpy(), cm[:C].cpu().numpy(), st


@pytest.mark.parametrize("greedy", [True, False], ids=["rounds-greedy", "empty"])
def test_batch_same_as_the_oracle_graph_by_graph(greedy):
    b = synth.batch_graphs(96, seed=41, nr_lo=10, nr_hi=4000, mu_lo=1.5, mu_hi=8.0)
    w_rm, w_cm, w_st = oracle_batch_det(b, greedy)
    rm, cm, st = run_batch_det(b, greedy)
    np.testing.assert_array_equal(rm, w_rm)
    np.testing.assert_array_equal(cm, w_cm)
    # the batch reports phases, levels, ... summed over its graphs; roots are not counted there
    assert {k: st[k] for k in STATS if k != "roots"} == {k: v for k, v in w_st.items() if k != "roots"}


@pytest.mark.parametrize("block,per_sm", [(64, 0), (256, 1), (1024, 1)])
def test_batch_same_for_every_geometry(block, per_sm):
    b = synth.batch_graphs(48, seed=42, nr_lo=10, nr_hi=6000)
    w_rm, w_cm, _ = oracle_batch_det(b, True)
    rm, cm, _ = run_batch_det(b, True, block_size=block, blocks_per_sm=per_sm)
    np.testing.assert_array_equal(rm, w_rm)
    np.testing.assert_array_equal(cm, w_cm)


# ------------------------------------------------------------ served path
def served_requests():
    """Uniform and R-MAT requests of 50 to 20,000 rows (worker blocks), and one
    R-MAT request of about 700 k edges (above the default threshold: the
    single-graph kernel, beside the workers)."""
    rng = np.random.default_rng(77)
    out = []
    for i in range(24):
        nr = int(np.exp(rng.uniform(np.log(50), np.log(20000))))
        nc = max(1, int(round(nr * rng.uniform(0.8, 1.25))))
        mu = rng.uniform(3, 16)
        if i % 2 == 0:
            out.append(synth.uniform_graph(nr, nc, max(1, int(round(2 * mu - 1))), seed=3000 + i))
        else:
            n = max(nr, nc)
            out.append(synth.rmat_graph(int(np.ceil(np.log2(max(n, 2)))), int(n * mu), seed=3000 + i, n=n))
    out.append(synth.rmat_graph(17, 800_000, seed=3999))
    return out


def test_served_results_equal_the_oracle_alone_and_in_the_mix():
    from paper_1303_1379_gb300 import bmatch
    reqs = served_requests()
    want = []
    for g in reqs:
        rm0, cm0, _, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        rm, cm, card, _ = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0)
        want.append((rm, cm, card))
    assert reqs[-1].nnz >= 524_288

    def fetch(srv, rid, g):
        info = srv.wait(rid)
        assert info["state"] == bmatch.BM_REQ_DONE and info["status"] == 0
        rm = np.empty(g.n_rows, np.int32)
        cm = np.empty(g.n_cols, np.int32)
        srv.fetch(rid, rm, cm)
        srv.release(rid)
        return rm, cm, info["card"]

    with bmatch.Server(keep_results=1, pool_bytes=1 << 30, deterministic=1) as srv:
        for g, w in zip(reqs[:8] + reqs[-1:], want[:8] + want[-1:]):  # alone, one at a time
            rm, cm, card = fetch(srv, srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx), g)
            assert card == w[2]
            np.testing.assert_array_equal(rm, w[0])
            np.testing.assert_array_equal(cm, w[1])
        ids = [srv.submit(g.n_rows, g.n_cols, g.col_ptr, g.row_idx) for g in reqs]  # the mix
        for g, w, rid in zip(reqs, want, ids):
            rm, cm, card = fetch(srv, rid, g)
            assert card == w[2]
            np.testing.assert_array_equal(rm, w[0])
            np.testing.assert_array_equal(cm, w[1])
        st = srv.stats()
        assert st["exclusive_runs"] == 2 and st["pool_used"] == 0  # the large request, alone and in the mix


# ------------------------------------------------------------ cheap matching in rounds
@pytest.mark.parametrize("name", ["uniform-ragged", "rmat15", "rmat17-rcp", "stencil150"])
def test_cheap_matching_in_rounds_equals_the_oracle(name):
    from paper_1303_1379_gb300 import bmatch
    from helpers import to_dev
    g = graph(name)
    w_rm, w_cm, w_card, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    f_rm, f_cm, f_card, f_st = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, w_rm, w_cm)
    cp, ri = to_dev(g)
    for block in (128, 512, 1024):
        m = bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, deterministic=1, block_size=block)
        try:
            assert m.greedy() == w_card
            rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
            cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
            m.get_matching(rm, cm)
            np.testing.assert_array_equal(rm.cpu().numpy(), w_rm)
            np.testing.assert_array_equal(cm.cpu().numpy(), w_cm)
            res = m.match(rm, cm)  # cheap matching + search: the oracle's end to end
            assert res.card == f_card and {k: res.stats[k] for k in STATS} == f_st
            np.testing.assert_array_equal(rm.cpu().numpy(), f_rm)
        finally:
            m.close()


def test_full_size_cheap_matching_in_rounds():
    from paper_1303_1379_gb300 import bmatch
    from helpers import to_dev
    g = synth.workload("rmat21")
    w_rm, _, w_card, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    cp, ri = to_dev(g)
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, deterministic=1) as m:
        assert m.greedy() == w_card
        rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
        m.get_matching(rm, None)
        np.testing.assert_array_equal(rm.cpu().numpy(), w_rm)


def test_batch_apsb_same_as_the_oracle():
    b = synth.batch_graphs(40, seed=43, nr_lo=10, nr_hi=3000)
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    w_rm = np.full(R, -1, np.int32)
    for k in range(b.n_graphs):
        g = b.graph(k)
        rm0, cm0, _, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        rm, _, _, _ = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0, apsb=True)
        w_rm[b.row_off[k]:b.row_off[k + 1]] = rm
    rm, _, _ = run_batch_det(b, True, mode=1)
    np.testing.assert_array_equal(rm, w_rm)


def test_match_host_buffers_deterministic():
    # bm_match_host (host CSR and start, copies inside the call) under the option
    from paper_1303_1379_gb300 import bmatch
    g = graph("rmat15")
    rm0, cm0 = start(g, "greedy")
    w_rm, w_cm, w_card, _ = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0)
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, None, None, deterministic=1) as m:
        h_rm, h_cm = rm0.copy(), cm0.copy()
        res = m.match_host(g.col_ptr, g.row_idx, h_rm, h_cm)
        assert res.card == w_card
        np.testing.assert_array_equal(h_rm, w_rm)
        np.testing.assert_array_equal(h_cm, w_cm)
