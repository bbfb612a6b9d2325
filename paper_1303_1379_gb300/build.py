"""Builds the CUDA library in-tree (sm_103a only): libbmatch.so and its
range-checked twin libbmatch_checked.so (compiled with BM_CHECKED: every
index the kernels compute from data is checked before use and an index out
of range, or an inconsistent matching between phases, is reported as
BM_ERR_CHECK instead of being used).  The two are compiled in parallel.

``nvcc -gencode arch=compute_103a,code=sm_103a`` cross-compiles without a GPU.
The library links the shared CUDA runtime, so inside a PyTorch process it
shares the runtime PyTorch already loaded.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libbmatch.so")
LIB_CHECKED = os.path.join(HERE, "libbmatch_checked.so")
SOURCES = [os.path.join(CSRC, f) for f in ("bmatch.cu", "bm_batch.cu", "bm_server.cu")]
DEPENDS = SOURCES + [os.path.join(CSRC, f) for f in ("bm_device.cuh", "bm_internal.h", "bm_pool.h")] + \
    [os.path.join(INCLUDE, "bmatch.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def cuda_lib_dir() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "lib64")


def is_stale(path: str = LIB) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in DEPENDS)


def _command(out: str, checked: bool, verbose: bool):
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-I", INCLUDE, "-shared",
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-cudart", "shared",
           "-Xlinker", "-rpath," + cuda_lib_dir(), *SOURCES, "-o", out + ".tmp"]
    if checked:
        cmd.insert(1, "-DBM_CHECKED")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def build(force: bool = False, verbose: bool = False, checked: bool | None = None) -> str:
    """Builds the stale libraries (both by default; checked=False / True: only
    the normal / the range-checked one).  Returns the normal library's path."""
    todo = []
    for path, chk in ((LIB, False), (LIB_CHECKED, True)):
        if checked is not None and chk != checked:
            continue
        if force or is_stale(path):
            todo.append((path, chk))
    procs = [(path, subprocess.Popen(_command(path, chk, verbose), stdout=subprocess.PIPE,
                                     stderr=subprocess.PIPE, text=True)) for path, chk in todo]
    errors = []
    for path, pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"nvcc failed for {os.path.basename(path)}:\n{out}{err}")
        else:
            os.replace(path + ".tmp", path)
            if verbose:
                print(err)
    if errors:
        raise RuntimeError("\n".join(errors))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
