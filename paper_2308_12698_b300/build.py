"""Builds libquadsim.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libquadsim.so")
#: the same sources with the kernels' device bounds checks compiled in (QS_CHECKED)
LIB_CHECKED = os.path.join(HERE, "libquadsim_checked.so")
SOURCES = [os.path.join(CSRC, f) for f in ("quadsim.cu", "model_fwd.cuh", "model_adj.cuh", "step_kernel.cuh",
                                           "vehicles.cuh", "adjoint_kernel.cuh", "collide.cuh", "compact.cuh",
                                           "checks.cuh", "stats.cuh")] + \
    [os.path.join(ROOT, "include", "quadsim.h")]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile libquadsim.so (and, with checked, libquadsim_checked.so beside it, in parallel)
    when a source is newer; returns the product library's path."""
    newest = max(os.path.getmtime(s) for s in SOURCES)
    targets = [(LIB, [])] + ([(LIB_CHECKED, ["-DQS_CHECKED"])] if checked else [])
    jobs = []
    for lib, extra in targets:
        if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
            continue
        cmd = [nvcc(), *NVCC_FLAGS, *extra, os.path.join(CSRC, "quadsim.cu"), "-o", lib + ".tmp"]
        if verbose and lib == LIB:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((lib, subprocess.Popen(cmd)))
    for lib, proc in jobs:
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, f"nvcc -> {lib}")
    for lib, _ in jobs:
        os.replace(lib + ".tmp", lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
