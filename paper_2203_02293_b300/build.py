"""Compile the CUDA library (librt.so) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "librt.so")
# the same library with every main device-memory access range-checked
# (RT_BOUNDS_CHECK): out-of-range accesses are counted and skipped
LIB_BOUNDS = os.path.join(HERE, "librt_bounds.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("rt_kernels.cu", "rt_api.cpp", "rt_noalloc.cu")]
HEADERS = [os.path.join(HERE, "csrc", "rt_internal.h"), os.path.join(ROOT, "include", "rt.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in SOURCES + HEADERS)


def build(lib: str = LIB, extra: list[str] | None = None, verbose: bool = False) -> str:
    """nvcc -O3 -lineinfo, static cudart, position-independent shared object."""
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", lib, *SOURCES, *(extra or [])]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    return lib


def build_bounds(lib: str = LIB_BOUNDS) -> str:
    """The bounds-check variant of the library."""
    return build(lib, extra=["-DRT_BOUNDS_CHECK"])


if __name__ == "__main__":
    print(build(verbose=True))
    print(build_bounds())
