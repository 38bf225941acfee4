"""Builds the CUDA library in-tree for sm_103a (GB300): libconvex_barrier.so next to this file."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "csrc", f) for f in ("convex_barrier.cu", "noalloc.cu", "tc_gemm.cu",
                                                           "ibounds.cu", "bab.cu", "state.cu")]
LIB = os.path.join(HERE, "libconvex_barrier.so")
OBJDIR = os.path.join(HERE, "_build")
DEPS = [os.path.join(HERE, "csrc", f) for f in
        ("convex_barrier.cu", "cb_common.cuh", "cb_kernels.cuh", "cb_backward.cuh", "cb_team.cuh",
         "cb_host_extra.inc", "noalloc.cu", "cb_walk.cuh", "cb_tc.cuh", "tc_gemm.cu", "cb_bf16.inc",
         "ibounds.cu", "bab.cu", "state.cu")] + \
    [os.path.join(HERE, "..", "include", "convex_barrier.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the translation units in parallel (nvcc -c), then links the shared library."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    procs = []
    for src in SRCS:
        obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
        cmd = [nvcc(), *NVCC_FLAGS, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd), obj, cmd))
    objs = []
    for p, obj, cmd in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, cmd)
        objs.append(obj)
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
