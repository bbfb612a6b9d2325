"""Batched matching (one persistent launch over many graphs) against the
oracle: every graph's |M| equals Hopcroft-Karp's, and each graph's slice of
the batch matching is valid and carries a Koenig certificate."""
import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import bmatch, synth

from helpers import VARIANTS, assert_maximum, vname

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_batch(b, greedy=True, init=None, **options):
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    rm = torch.full((max(R, 1),), -1, dtype=torch.int32, device="cuda")
    cm = torch.full((max(C, 1),), -1, dtype=torch.int32, device="cuda")
    if init is not None:
        rm[:R] = torch.from_numpy(init[0]).cuda()
        cm[:C] = torch.from_numpy(init[1]).cuda()
    card = torch.zeros(max(b.n_graphs, 1), dtype=torch.int32, device="cuda")
    with bmatch.Batch.from_synth(b, **options) as bb:
        rc, st = bb.match(rm, cm, greedy=greedy, card_out=card)
        status, phases = bb.graph_status()
    assert rc == 0 and np.all(status == 0)
    return rm[:R].cpu().numpy(), cm[:C].cpu().numpy(), card[:b.n_graphs].cpu().numpy(), st


def check_all(b, rm, cm, card, want):
    for k in range(b.n_graphs):
        g = b.graph(k)
        r = rm[b.row_off[k]:b.row_off[k + 1]]
        c = cm[b.col_off[k]:b.col_off[k + 1]]
        assert card[k] == want[k], k
        assert_maximum(g, r, c, int(card[k]), int(want[k]))


@pytest.mark.parametrize("variant", VARIANTS[:6], ids=vname)
def test_batch_matches_oracle(variant):
    b = synth.batch_graphs(97, seed=31, nr_lo=20, nr_hi=3000)
    _, _, want = oracle.hk_batch(b, greedy_first=False)
    v = {k: x for k, x in variant.items() if k != "driver"}
    rm, cm, card, st = run_batch(b, greedy=True, **v)
    check_all(b, rm, cm, card, want)
    assert st["phases"] >= b.n_graphs


@pytest.mark.parametrize("block", [64, 256, 1024])
def test_batch_launch_geometry_and_empty_start(block):
    b = synth.batch_graphs(64, seed=5, nr_lo=1, nr_hi=5000, mu_lo=1.0, mu_hi=6.0)
    _, _, want = oracle.hk_batch(b, greedy_first=False)
    rm, cm, card, _ = run_batch(b, greedy=False, block_size=block)
    check_all(b, rm, cm, card, want)


def test_batch_from_given_matching_and_replay():
    """Initial matchings from the oracle's greedy, two replays of the recorded
    launch: same cardinalities both times."""
    b = synth.batch_graphs(40, seed=8, nr_lo=100, nr_hi=20000)
    rm0 = np.full(int(b.row_off[-1]), -1, np.int32)
    cm0 = np.full(int(b.col_off[-1]), -1, np.int32)
    for k in range(b.n_graphs):
        g = b.graph(k)
        r, c, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        rm0[b.row_off[k]:b.row_off[k + 1]] = r
        cm0[b.col_off[k]:b.col_off[k + 1]] = c
    _, _, want = oracle.hk_batch(b, greedy_first=True)
    R, C = len(rm0), len(cm0)
    with bmatch.Batch.from_synth(b) as bb:
        for _ in range(2):
            rm = torch.from_numpy(rm0).cuda()
            cm = torch.from_numpy(cm0).cuda()
            card = torch.zeros(b.n_graphs, dtype=torch.int32, device="cuda")
            bb.match(rm, cm, greedy=False, card_out=card)
            check_all(b, rm.cpu().numpy(), cm.cpu().numpy(), card.cpu().numpy(), want)


def test_batch_autotune_picks_a_working_geometry():
    b = synth.batch_graphs(128, seed=9, nr_lo=100, nr_hi=8000)
    _, _, want = oracle.hk_batch(b, greedy_first=False)
    R, C = int(b.row_off[-1]), int(b.col_off[-1])
    rm0 = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    cm0 = torch.full((C,), -1, dtype=torch.int32, device="cuda")
    rmw, cmw = torch.empty_like(rm0), torch.empty_like(cm0)
    with bmatch.Batch.from_synth(b) as bb:
        best, ms = bb.autotune(rm0, cm0, rmw, cmw, [(256, 2), (512, 2), (1024, 1)])
        assert 0 <= best < 3 and ms[best] > 0 and ms[best] == min(m for m in ms if m > 0)
        rm, cm = rm0.clone(), cm0.clone()
        card = torch.zeros(b.n_graphs, dtype=torch.int32, device="cuda")
        bb.match(rm, cm, greedy=True, card_out=card)
    check_all(b, rm.cpu().numpy(), cm.cpu().numpy(), card.cpu().numpy(), want)


def test_batch_rejects_invalid_graph():
    b = synth.batch_graphs(10, seed=2, nr_lo=50, nr_hi=100)
    bad = b.row_idx.copy()
    bad[5] = 10_000_000
    with pytest.raises(bmatch.BMError) as e:
        bmatch.Batch(b.n_rows, b.n_cols, b.row_off, b.col_off, b.edge_off, b.col_ptr, bad)
    assert e.value.status == bmatch.BM_ERR_INVALID_CSR


@pytest.mark.slow
def test_batch_full_size_4096_graphs():
    """The batched workload at full size, in the launch geometry the benchmark's
    autotuner settles on (512 threads, 2 blocks per SM) with the cheap matching
    inside the launch.  The workload is 4,096 graphs, 226 M edges, rows
    log-uniform in [100, 50,000], seed 3.  Every graph's |M| equals
    Hopcroft-Karp's, and every graph's slice of the batch matching is valid and
    carries a Koenig certificate."""
    b = synth.batch_graphs(4096, seed=3)
    _, _, want = oracle.hk_batch(b, greedy_first=True)
    rm, cm, card, st = run_batch(b, greedy=True, block_size=512, blocks_per_sm=2)
    assert np.array_equal(card, want)
    check_all(b, rm, cm, card, want)
