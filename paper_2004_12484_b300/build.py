"""Build step of the CUDA library: compiles the ``csrc`` sources for sm_103a into
``libenuf.so`` inside the package directory (in-tree, so that the built
library travels with the source tree).

    python -m paper_2004_12484_b300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libenuf.so")
# the benchmark's FMA-rate probe, kept out of the library
PROBE_LIB = os.path.join(HERE, "libenuf_probe.so")
# the same library with bounds checks in every kernel (tests only)
CHECK_LIB = os.path.join(HERE, "libenuf_check.so")
HEADER = os.path.join(ROOT, "include", "enuf.h")

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
    "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-O3",
]


def _sources():
    out = [HEADER, os.path.join(ROOT, "include", "enuf_probe.h")]
    for f in sorted(os.listdir(SRC_DIR)):
        if f.endswith((".cu", ".cuh")):
            out.append(os.path.join(SRC_DIR, f))
    return out


def needs_build() -> bool:
    for lib in (LIB, PROBE_LIB, CHECK_LIB):
        if not os.path.exists(lib):
            return True
        t = os.path.getmtime(lib)
        if any(os.path.getmtime(s) > t for s in _sources()):
            return True
    return False


def nvcc() -> str:
    for cand in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"]:
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    srcs = [os.path.join(SRC_DIR, "enuf.cu"), os.path.join(SRC_DIR, "noalloc.cu"), os.path.join(SRC_DIR, "mlp.cu")]
    jobs = [
        (LIB, [*NVCC_FLAGS, *srcs]),
        (PROBE_LIB, [*NVCC_FLAGS, os.path.join(SRC_DIR, "probe.cu")]),
        (CHECK_LIB, [*NVCC_FLAGS, "-DENUF_BOUNDS_CHECK", *srcs]),
    ]
    # the libraries compile side by side
    procs, cmds = [], []
    for lib, args in jobs:
        c = [nvcc(), *args, "-o", lib + f".tmp{os.getpid()}"]
        if verbose:
            print(" ".join(c), flush=True)
        cmds.append(c)
        procs.append(subprocess.Popen(c))
    rcs = [pr.wait() for pr in procs]
    for c, rc in zip(cmds, rcs):
        if rc != 0:
            raise subprocess.CalledProcessError(rc, c)
    for lib, _ in jobs:
        os.replace(lib + f".tmp{os.getpid()}", lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
