"""bench.py matches the committed ncu counters to the persistent kernel by a
hash of its code.  Comment and whitespace edits must keep the hash; any code
edit must change it (then the traffic figure is dropped as stale)."""
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

