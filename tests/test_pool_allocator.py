"""The matching server's pool bookkeeping (csrc/bm_pool.h), compiled with the
host C++ compiler and driven through random allocate / release sequences:
extents never overlap and stay inside the pool, the byte count is exact, and
releasing everything coalesces the pool back into one free extent."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1303_1379_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include "bm_pool.h"

static unsigned long long state = 88172645463325252ull;
static unsigned long long next_u() { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return state; }

struct Ext { std::size_t off, bytes; };

int main() {
    for (int trial = 0; trial < 50; ++trial) {
        const std::size_t size = (1 + next_u() % 4096) * 1000 + next_u() % 999;
        bms::PoolAllocator a(size);
        const std::size_t cap = size & ~std::size_t(255);
        if (a.size() != cap) { std::printf("size %zu %zu\n", a.size(), cap); return 1; }
        std::vector<Ext> live;
        std::size_t want_used = 0;
        for (int op = 0; op < 2000; ++op) {
            if (live.empty() || next_u() % 3 != 0) {
                const std::size_t b = 1 + next_u() % (cap / 8 + 1);
                std::size_t off = 0;
                if (a.alloc(b, &off)) {
                    const std::size_t r = (b + 255) & ~std::size_t(255);
                    if (off % 256 != 0 || off + r > cap) { std::printf("bounds\n"); return 1; }
                    live.push_back({off, b});
                    want_used += r;
                }
            } else {
                const std::size_t k = next_u() % live.size();
                a.release(live[k].off, live[k].bytes);
                want_used -= (live[k].bytes + 255) & ~std::size_t(255);
                live.erase(live.begin() + k);
            }
            if (a.used() != want_used) { std::printf("used %zu %zu\n", a.used(), want_used); return 1; }
            std::vector<Ext> s = live;
            std::sort(s.begin(), s.end(), [](const Ext& x, const Ext& y) { return x.off < y.off; });
            for (std::size_t i = 1; i < s.size(); ++i)
                if (s[i - 1].off + ((s[i - 1].bytes + 255) & ~std::size_t(255)) > s[i].off) { std::printf("overlap\n"); return 1; }
        }
        for (const Ext& e : live) a.release(e.off, e.bytes);
        std::size_t off = 1;
        if (a.used() != 0 || !a.alloc(cap, &off) || off != 0) { std::printf("coalesce\n"); return 1; }
    }
    std::printf("ok\n");
    return 0;
}
"""


def test_pool_allocator_random_sequences(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "pool_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "pool_driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
