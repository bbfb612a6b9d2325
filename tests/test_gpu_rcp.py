"""Parity on randomly permuted graphs (Section 4's RCP instances).

Section 4 permutes the rows and columns of every matrix at random; the
searches then take completely different paths (on the 2000 x 2000 mesh, 8
phases and a few thousand BFS levels instead of about 70 phases and 100,000
levels), which the paper finds harder for most algorithms.  The CUDA path
must still reach Hopcroft-Karp's |M| with a matching that carries a Koenig
certificate, from the oracle's column-order greedy start and from the GPU's
own cheap matching.
"""
import numpy as np
import pytest

import oracle
from paper_1303_1379_gb300 import bmatch, synth

from helpers import VARIANTS, assert_maximum, gpu_match, oracle_max, to_dev, vname

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAPHS = {
    "rmat18-rcp": lambda: synth.permute_graph(synth.rmat_graph(18, 1 << 22, seed=1), seed=5),
    "stencil500-rcp": lambda: synth.workload("stencil500-rcp"),
    "uniform-rcp": lambda: synth.permute_graph(synth.uniform_graph(300_007, 299_993, 5, seed=8), seed=5),
}
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        _cache[name] = (g, oracle_max(g))
    return _cache[name]


def test_permutation_changes_the_graph_not_its_maximum():
    g = synth.workload("stencil500")
    h, want = graph("stencil500-rcp")
    assert h.nnz == g.nnz and not np.array_equal(h.col_ptr, g.col_ptr)
    assert want == oracle_max(g)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("variant", [VARIANTS[0], VARIANTS[1], VARIANTS[2], VARIANTS[3]], ids=vname)
def test_permuted_graphs_from_the_oracle_greedy(name, variant):
    g, want = graph(name)
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    rm, cm, card, st = gpu_match(g, (rm0, cm0), **variant)
    assert_maximum(g, rm, cm, card, want)
    assert st["initial_card"] == int((cm0 >= 0).sum())


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("variant", [VARIANTS[0], VARIANTS[1]], ids=vname)
def test_permuted_graphs_from_the_gpu_cheap_matching(name, variant):
    """The setting the benchmark times: the GPU cheap matching, then the search."""
    g, want = graph(name)
    cp, ri = to_dev(g)
    rm = torch.empty(g.n_rows, dtype=torch.int32, device="cuda")
    cm = torch.empty(g.n_cols, dtype=torch.int32, device="cuda")
    with bmatch.Matcher(g.n_rows, g.n_cols, g.nnz, cp, ri, **variant) as m:
        m0 = m.greedy()
        res = m.match(rm, cm)
    assert res.stats["initial_card"] == m0 <= want
    assert_maximum(g, rm.cpu().numpy(), cm.cpu().numpy(), res.card, want)
