"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point include/bmatch.h declares, and the ctypes structs have the C
layout."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1303_1379_gb300 import bmatch, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        names += re.findall(r"^BM_API\s+[\w\s\*]+?\b(bm_\w+)\s*\(", text, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    lib = bmatch.load()
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\sT\s+(\w+)", out.stdout))
        assert set(names) <= exported
    assert set(bmatch.EXPORTS) <= set(names)


def test_checked_library_exports_the_same_symbols():
    """The range-checked twin (BM_CHECKED) is built beside the library and
    exports the same entry points, so BMATCH_CHECKED=1 can swap it in."""
    build.build(checked=True)
    assert os.path.exists(build.LIB_CHECKED)
    names = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_CHECKED], capture_output=True, text=True)
    if out.returncode == 0:
        assert set(names) <= set(re.findall(r"\sT\s+(\w+)", out.stdout))
    lib = ctypes.CDLL(build.LIB_CHECKED)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults():
    assert bmatch.status_string(0) == "ok"
    for code in range(-11, 2):
        assert bmatch.status_string(code) != "unknown status"
    o = bmatch.default_options()
    assert (o.mode, o.bfs, o.driver, o.wr_one_endpoint, o.max_phases) == (0, 1, 0, 1, 0)
    assert bmatch.load().bm_version() >= 10000


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "bmatch.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(bm_options), offsetof(bm_options, wait_timeout_ns),
         sizeof(bm_stats), offsetof(bm_stats, levels), offsetof(bm_stats, fix_repairs),
         offsetof(bm_options, total_timeout_ns));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(bmatch.bm_options), bmatch.bm_options.wait_timeout_ns.offset,
            ctypes.sizeof(bmatch.bm_stats), bmatch.bm_stats.levels.offset,
            bmatch.bm_stats.fix_repairs.offset, bmatch.bm_options.total_timeout_ns.offset]
    assert got == want


def test_header_is_c_compatible(tmp_path):
    src = tmp_path / "use.c"
    src.write_text('#include "bmatch.h"\nint f(bm_ctx* c){ return bm_match(c, 0, 0, 0, 0); }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(tmp_path / "use.o")], check=True)


def test_binding_rejects_bad_buffers():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        bmatch._ptr(torch.zeros(4, dtype=torch.int64))
    with pytest.raises(TypeError):
        bmatch._ptr(torch.zeros(8, dtype=torch.int32)[::2])


def test_deterministic_option_is_checked_before_any_device_call():
    # bm_create checks its options first: an invalid deterministic setting
    # (a value other than 0/1, or a variant the option does not cover) is
    # refused with BM_ERR_INVALID_ARG without touching a GPU.
    lib = bmatch.load()
    ctx = ctypes.c_void_p()
    bad = [dict(deterministic=2), dict(deterministic=1, driver=1), dict(deterministic=1, bfs=0),
           dict(deterministic=1, wr_one_endpoint=0)]
    for kw in bad:
        o = bmatch.default_options(**kw)
        rc = lib.bm_create(10, 10, 0, None, None, None, ctypes.byref(o), ctypes.byref(ctx))
        assert rc == bmatch.BM_ERR_INVALID_ARG, kw
        assert not ctx.value
