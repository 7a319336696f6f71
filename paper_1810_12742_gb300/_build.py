"""Build libhines.so in-tree for sm_103a (nvcc + g++, no cmake).

Each translation unit compiles in parallel into ``_build/``; the shared
library is linked with the static CUDA runtime.  A content hash of the
sources and flags skips rebuilds that would change nothing.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhines.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3"] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: libhines needs the CUDA toolkit to build")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return sorted(hs + [os.path.join(ROOT, "include", "hines.h")])


def _digest(extra=()) -> str:
    h = hashlib.sha256()
    for f in _sources() + _headers():
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS + list(extra)).encode())
    return h.hexdigest()


# The files that decide what the task kernels k_units<...> do and how the
# solves launch them: their code, the plan structure they read, the planner
# that builds the schedule and the entry points that size the grid.  DRAM
# counters taken on these files stay valid while none of them changes.
UNIT_KERNEL_FILES = ("csrc/unit_kernels.cuh", "csrc/unit_kernels_p1.cu", "csrc/unit_kernels_p2.cu",
                     "csrc/unit_dispatch.cu", "csrc/device_common.cuh", "csrc/kernels.h", "csrc/plan.h",
                     "csrc/plan.cpp", "csrc/hines_abi.cu")


def unit_kernel_digest() -> str:
    h = hashlib.sha256()
    for rel in UNIT_KERNEL_FILES:
        h.update(rel.encode())
        with open(os.path.join(PKG, rel), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libhines.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()
    jobs = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
        else:
            cmd = ["g++", *CXX_FLAGS, "-c", src, "-o", obj]
        jobs.append((cmd, obj))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, [c for c, _ in jobs]))
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, "-shared", *ARCH, "-o", tmp, *[o for _, o in jobs], "-cudart", "static"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
