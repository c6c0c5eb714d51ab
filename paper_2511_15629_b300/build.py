"""Build the CUDA library libesdp.so in-tree (nvcc, sm_103a only)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libesdp.so")
# the same sources with per-phase cycle counters in the sweep (a measurement build)
LIB_PHASE = os.path.join(HERE, "libesdp_phase.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.h")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def build(force: bool = False, verbose: bool = False, phase_clocks: bool = False) -> str:
    """Compile libesdp.so (or, with phase_clocks, libesdp_phase.so: the sweep
    with per-phase clock counters, read by esdp_phase_clocks)."""
    lib = LIB_PHASE if phase_clocks else LIB
    if not force and not stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *sources()]
    if phase_clocks:
        cmd.insert(1, "-DESDP_PHASE_CLOCKS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                phase_clocks="--phase-clocks" in sys.argv))
