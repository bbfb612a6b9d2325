"""Builds the CUDA library libbmatch.so in-tree (sm_103a only).

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


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in DEPENDS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not is_stale():
        return LIB
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-I", INCLUDE, "-shared",
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-cudart", "shared",
           "-Xlinker", "-rpath," + cuda_lib_dir(), *SOURCES, "-o", LIB + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
