"""The range-checked build on the GPU.

libbmatch_checked.so (compiled with BM_CHECKED) checks every index the kernels
compute from data -- row ids, matched columns, roots, queue entries,
predecessors -- before using it, and between phases checks that rmatch and
cmatch are mutual inverses; a violation returns BM_ERR_CHECK.  It stands in
for a memory checker (compute-sanitizer is closed on this machine).  These tests
run the parity workloads of every variant (the deterministic option too, whose
matching must be the oracle's), the batched path and the allocation-free entry
point through it, in a fresh process (the library is
chosen at the first load), and require the oracle's |M| with no check firing.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch
import oracle
from paper_1303_1379_gb300 import bmatch, build, synth
from helpers import VARIANTS, gpu_match, assert_maximum, oracle_max
assert bmatch.library_path() == build.LIB_CHECKED
out = []
graphs = {
    "uniform": synth.uniform_graph(7919, 8111, 5, seed=21),
    "rmat15": synth.rmat_graph(15, 200000, seed=5),
    "stencil150": synth.stencil_graph(150, 2250, 0.05, seed=6),
    "rmat16-rcp": synth.permute_graph(synth.rmat_graph(16, 1 << 20, seed=2), seed=5),
}
for name, g in graphs.items():
    want = oracle_max(g)
    rm0, cm0, _ = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
    for v in VARIANTS:
        rm, cm, card, st = gpu_match(g, (rm0, cm0), **v)
        assert_maximum(g, rm, cm, card, want)
        out.append([name, v, card, st["status"]])
    for apsb in (0, 1):  # the deterministic option: the oracle's exact matching
        w_rm, w_cm, _, _ = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0, apsb=bool(apsb))
        rm, cm, card, st = gpu_match(g, (rm0, cm0), deterministic=1, mode=apsb)
        assert np.array_equal(rm, w_rm) and np.array_equal(cm, w_cm)
        out.append([name, {"deterministic": 1, "mode": apsb}, card, st["status"]])
# batched path
b = synth.batch_graphs(64, seed=3)
bb = bmatch.Batch.from_synth(b)
R, C = int(b.row_off[-1]), int(b.col_off[-1])
rm = torch.full((R,), -1, dtype=torch.int32, device="cuda")
cm = torch.full((C,), -1, dtype=torch.int32, device="cuda")
card = torch.zeros(b.n_graphs, dtype=torch.int32, device="cuda")
rc, st = bb.match(rm, cm, greedy=True, card_out=card)
_, _, want = oracle.hk_batch(b, greedy_first=True)
assert rc == 0 and np.array_equal(card.cpu().numpy(), want)
out.append(["batch64", None, int(card.sum()), st["status"]])
bd = bmatch.Batch.from_synth(b, deterministic=1)
rm.fill_(-1); cm.fill_(-1)
rc, st = bd.match(rm, cm, greedy=True)
w_rm = np.full(R, -1, np.int32)
for k in range(b.n_graphs):
    gk = b.graph(k)
    g_rm, g_cm, _, _ = oracle.greedy_rounds(gk.n_rows, gk.n_cols, gk.col_ptr, gk.row_idx)
    w_rm[b.row_off[k]:b.row_off[k + 1]] = oracle.apfb_wr_det(gk.n_rows, gk.n_cols, gk.col_ptr, gk.row_idx, g_rm, g_cm)[0]
assert rc == 0 and np.array_equal(rm.cpu().numpy(), w_rm)
out.append(["batch64-deterministic", None, int((cm >= 0).sum()), st["status"]])
# allocation-free entry point
g = graphs["rmat15"]
cp = torch.from_numpy(g.col_ptr).cuda(); ri = torch.from_numpy(g.row_idx).cuda()
r0 = torch.full((g.n_rows,), -1, dtype=torch.int32, device="cuda")
c0 = torch.full((g.n_cols,), -1, dtype=torch.int32, device="cuda")
rc, c = bmatch.bm_match_noalloc(g.n_rows, g.n_cols, g.nnz, cp, ri, r0, c0)
assert rc == 0 and c == oracle_max(g), (rc, c)
out.append(["noalloc", None, c, rc])
print("RESULT " + json.dumps(out))
'''


def test_checked_build_runs_every_variant_without_a_check_firing():
    from paper_1303_1379_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, BMATCH_CHECKED="1")
    res = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    line = [l for l in res.stdout.splitlines() if l.startswith("RESULT ")][-1]
    rows = json.loads(line[7:])
    assert len(rows) == 4 * (8 + 2) + 3
    assert all(r[3] == 0 for r in rows)
