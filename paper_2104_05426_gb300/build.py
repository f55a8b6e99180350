"""In-tree build of libjefi.so for sm_103a (nvcc for the kernels, g++ for the host library).

Objects go to ``_build/`` next to this file and the shared library to
``libjefi.so``; both are git-ignored.  Translation units compile in
parallel.  Host code is compiled with ``-ffp-contract=off`` because the
exact FP64 slot rule must not be contracted into fused multiply-adds.
"""
from __future__ import annotations

import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libjefi.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
             "-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(CUDA_HOME, "include")]

CU_SOURCES = ["jefi_kernels.cu", "jefi_staged.cu", "jefi_staged_b32_48.cu", "jefi_staged_b64_96.cu",
              "jefi_noalloc.cu"]
CXX_SOURCES = ["jefi_host.cpp"]
HEADERS = ["jefi_internal.h", "jefi_device.cuh", "jefi_staged.cuh"]
_lock = threading.Lock()


def _sources():
    return ([os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES + HEADERS]
            + [os.path.join(INCLUDE, "jefi.h")])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit and link libjefi.so; returns its path."""
    with _lock:
        if not force and up_to_date():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        jobs, objs = [], []
        for f in CU_SOURCES:
            o = os.path.join(BUILD, f + ".o")
            jobs.append([NVCC, *NVCC_FLAGS, "-c", os.path.join(CSRC, f), "-o", o])
            objs.append(o)
        for f in CXX_SOURCES:
            o = os.path.join(BUILD, f + ".o")
            jobs.append(["g++", *CXX_FLAGS, "-c", os.path.join(CSRC, f), "-o", o])
            objs.append(o)
        procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
        errors = []
        for j, p in zip(jobs, procs):
            out, _ = p.communicate()
            if verbose and out:
                print(out.decode(errors="replace"))
            if p.returncode != 0:
                errors.append(" ".join(j) + "\n" + out.decode(errors="replace"))
        if errors:
            raise RuntimeError("libjefi build failed:\n" + "\n".join(errors))
        tmp = LIB + f".tmp{os.getpid()}"
        link = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("libjefi link failed:\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
