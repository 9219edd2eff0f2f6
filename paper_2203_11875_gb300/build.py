"""Build the in-tree C-ABI library ``libcondipm.so`` for sm_103a.

Each translation unit is compiled in parallel with nvcc (host C++ with g++),
then linked into one shared library next to this file.  A content hash of the
sources and flags is stored beside the library, so an unchanged tree is not
rebuilt.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libcondipm.so")
BUILD_DIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC"]
CU_SOURCES = ["kernels_model.cu", "kernels_linalg.cu", "kernels_trsm.cu", "api.cu", "kkt.cu", "ipm.cu", "sens.cu", "batch.cu", "noalloc.cu", "peak.cu", "fullspace.cu"]
CXX_SOURCES = ["plan.cpp", "fsplan.cpp"]
HEADERS = ["common.cuh", "plan.h", "fsplan.h", "opf_handle.h", "internal.h"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcondipm.so")


def _digest() -> str:
    h = hashlib.sha256()
    for f in CU_SOURCES + CXX_SOURCES + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(ROOT, "include", "condipm.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link libcondipm.so; returns its path."""
    stamp = LIB + ".sha256"
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD_DIR, f.replace(".cu", ".o"))
        jobs.append([nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD_DIR, f.replace(".cpp", ".o"))
        jobs.append([os.environ.get("CXX", "g++"), *CXX_FLAGS, "-c", os.path.join(CSRC, f), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"compilation failed: {cmd[-3]}")
        return cmd[-1]

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
