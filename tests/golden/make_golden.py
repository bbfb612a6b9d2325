"""Writes tests/golden/workloads.txt: the maximum matching size of each
benchmark workload, computed by the oracle only (greedy start + Hopcroft-Karp,
checked by the Koenig certificate), and the result of the deterministic
option's rules from the empty matching (the cheap matching in proposal rounds,
then the search level by level): its phases, levels and a SHA-256 prefix of
the row-to-column array (int32, little-endian).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1303_1379_gb300 import synth  # noqa: E402


def main():
    lines = ["# name  nnz  greedy (oracle's column-order cheap matching)  max (Hopcroft-Karp)",
             "#   det_*: proposal rounds + level-by-level search from the empty matching",
             "# written by tests/golden/make_golden.py (oracle only)"]
    for name in ("uniform10k", "rmat21", "stencil2000"):
        g = synth.workload(name)
        rm, cm, greedy = oracle.greedy(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        if name == "uniform10k":  # this workload starts from the empty matching
            rm, cm = oracle.empty_matching(g.n_rows, g.n_cols)
        rm, cm, card, phases = oracle.hopcroft_karp(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm)
        st, cover = oracle.konig(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm, cm)
        assert st == 0 and cover == card
        rm0, cm0, _, _ = oracle.greedy_rounds(g.n_rows, g.n_cols, g.col_ptr, g.row_idx)
        d_rm, _, d_card, d_st = oracle.apfb_wr_det(g.n_rows, g.n_cols, g.col_ptr, g.row_idx, rm0, cm0)
        assert d_card == card
        sha = hashlib.sha256(d_rm.astype("<i4").tobytes()).hexdigest()[:16]
        lines.append(f"{name} nnz={g.nnz} greedy={greedy} max={card} hk_phases={phases} "
                     f"det_phases={d_st['phases']} det_levels={d_st['levels']} det_rmatch_sha={sha}")
        print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
