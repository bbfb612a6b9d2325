"""bench.py's measurement helpers, on the CPU: the committed ncu counters are
matched to a kernel by a hash of its code (comment and whitespace edits keep
the hash, any code edit changes it and the traffic figure is dropped as
stale), and the roofline's byte counts follow their stated per-unit figures."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_comments_and_whitespace_do_not_count():
    b = _bench()
    code = "int f(int a) {\n    return a + 1;  // one more\n}\n"
    assert b._code_only(code) == b._code_only("/* header\n   block */ int  f(int a) { return a + 1; }")
    assert b._code_only(code) != b._code_only(code.replace("a + 1", "a + 2"))


def test_byte_model_follows_its_per_unit_figures():
    """The roofline's byte counts from a launch's counters, checked term by term
    against the per-unit figures the bench states (4-byte words, each counted
    once where it is read or written)."""
    b = _bench()
    st = {"phases": 3, "final_card": 50, "columns_expanded": 10, "edges_scanned": 100,
          "edges_to_matched": 60, "inserted": 7, "endpoints": 4, "alternate_steps": 9, "roots": 12}
    nr, nc = 200, 150
    levels_wr = 10 * (12 + 8) + 100 * 8 + 60 * 4 + 7 * 16 + 4 * 12
    levels_plain = 10 * 12 + 100 * 8 + 60 * 4 + 7 * 12 + 4 * 12
    assert b.level_bytes(st, True) == levels_wr
    assert b.level_bytes(st, False) == levels_plain
    per_phase = 12 * nc + (8 * nr + 4 * 50) + 4 * nr
    assert b.method_bytes(st, nr, nc, True) == levels_wr + 3 * per_phase + 9 * 20 + 4 * 4
    # one endpoint per root: one InitBfsArray, resets of inserted columns and carried roots,
    # record-based Alternate, no FixMatching
    assert b.performed_bytes(st, nr, nc, True, True) == levels_wr + 12 * nc + 16 * 7 + 20 * 12 + 16 * 9 + 8 * 4
    assert b.performed_bytes(st, nr, nc, False, False) == b.method_bytes(st, nr, nc, False)


def test_source_hash_tracks_each_kernel():
    b = _bench()
    h1, h2 = b.source_hash("k_match"), b.source_hash("k_batch")
    assert len(h1) == len(h2) == 16 and h1 != h2


def test_golden_lines_parse():
    """Every stored workload line parses (numbers and the deterministic
    option's array digest), as bench.py reads it."""
    b = _bench()
    for name in ("uniform10k", "rmat21", "stencil2000"):
        f = b.golden_fields(name)
        assert int(f["max"]) > 0 and int(f["det_phases"]) >= 1 and int(f["det_levels"]) >= 1
        assert len(f["det_rmatch_sha"]) == 16
        assert b.golden_max(name) == int(f["max"]) == b.golden_max(name + "-rcp")
