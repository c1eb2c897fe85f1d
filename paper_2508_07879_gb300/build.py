"""Build libqldpc.so in-tree: the sm_103a decoder kernels plus the C-ABI host code.

The kernel and host translation units compile in parallel and link into
``paper_2508_07879_gb300/libqldpc.so`` with the CUDA runtime linked statically, so loading the
library needs only the driver.  Objects go to ``paper_2508_07879_gb300/_build/``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqldpc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "-Xptxas", "-v", "--fmad=false"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-Wall", "-Wextra"]

KERNEL_SOURCES = ["msa_f32.cu", "msa_i16.cu", "msa_i8.cu", "msa_i16x2.cu", "msa_i8x2.cu", "msa_f32x2.cu", "msa_learned.cu",
                  "msa_layered.cu", "nms_train.cu", "server_f32.cu", "server_i16.cu", "server_i8.cu",
                  "qldpc_noalloc.cu"]
HOST_SOURCES = ["qldpc_host.cpp", "qldpc_server.cpp", "qldpc_learned.cpp"]
HEADERS = ["msa_launch.h", "msa_kernel.cuh", "msa_packed.cuh", "server_kernel.cuh", "graph.h"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libqldpc.so")
    return cand


def _cuda_include(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def _inputs():
    files = [os.path.join(CSRC, f) for f in KERNEL_SOURCES + HOST_SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "qldpc.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libqldpc.so if any source is newer than it.  Returns the library path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    for src in KERNEL_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(([nvcc, *ARCH, *NVCC_FLAGS, *inc, "-c", os.path.join(CSRC, src), "-o", obj], obj))
    cxx = shutil.which("g++") or "g++"
    for src in HOST_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(([cxx, *CXX_FLAGS, *inc, "-I" + _cuda_include(nvcc), "-c",
                      os.path.join(CSRC, src), "-o", obj], obj))

    def run(job):
        cmd, _ = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"compilation failed: {' '.join(cmd)}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for _, o in jobs]]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("link of libqldpc.so failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
