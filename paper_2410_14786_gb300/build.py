"""Build libbddc.so in-tree for sm_103a (nvcc + g++, translation units in parallel)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbddc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["bddc_kernels.cu", "bddc_bgemv_tma.cu", "bddc_pcg.cu", "coarse_solve.cu", "bddc_api.cu",
              "bddc_static_scratch.cu", "bddc_tc_gemm.cu"]
CXX_SOURCES = ["bddc_setup.cpp", "coarse_sparse.cpp"]
HEADERS = ["dense.hpp", "internal.hpp", "kernels.cuh", "sym_layout.hpp"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbddc")


def _cuda_include() -> str:
    nv = _nvcc()
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), "include")


def _inputs():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "bddc.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3",
                     "-Xptxas", "-O3", *inc, "-c", os.path.join(CSRC, f), "-o", o])
    for f in CXX_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-ffp-contract=fast", "-pthread",
                     "-I", _cuda_include(), *inc, "-c", os.path.join(CSRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"compile failed: {cmd[-3]}")
        return r

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
