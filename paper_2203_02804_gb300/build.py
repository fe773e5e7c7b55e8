"""Build the CUDA library in-tree: paper_2203_02804_gb300/libttprice.so (sm_103a only).

    python -m paper_2203_02804_gb300.build

Plain nvcc, one translation unit, no CMake.  Rebuilds only when a source is
newer than the library.  nvcc cross-compiles, so this also works on a machine
without a GPU.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libttprice.so")
SOURCES = ["ttprice.cu", "mlp.cu", "probe.cu"]
DEPS = ["ttprice.cu", "ttprice_device.cuh", "ttprice_kernels.cuh", "ttprice_tc.cuh", "mlp.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libttprice.so")
    return cand


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the sources to objects in parallel, then link the shared library."""
    deps = [os.path.join(CSRC, f) for f in DEPS] + [os.path.join(INCLUDE, h) for h in ("ttprice.h", "ttmlp.h", "ttprobe.h")]
    if not force and not _stale(LIB, deps):
        return LIB
    objs, procs = [], []
    for s in SOURCES:
        obj = os.path.join(CSRC, os.path.splitext(s)[0] + ".o")
        cmd = [nvcc_path(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-c", "-o", obj, os.path.join(CSRC, s)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    failed = [p.wait() for p in procs]
    if any(failed):
        raise subprocess.CalledProcessError(max(failed), "nvcc")
    tmp = LIB + ".tmp"
    subprocess.run([nvcc_path(), *ARCH, "-shared", "-o", tmp, *objs], check=True)
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
