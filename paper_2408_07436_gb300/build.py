"""Compile the CUDA library for sm_103a, in tree (``paper_2408_07436_gb300/libm2l_gb300.so``), and
the FMA-throughput probe the bench takes its CUDA-core peaks from (``libm2l_peaks.so``).

Each translation unit is compiled by nvcc in parallel, then linked into one shared library.
No CMake; the same command works on the x86 build container and on the Arm GPU host.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libm2l_gb300.so")
SOURCES = ["plan.cpp", "linalg.cpp", "capi.cpp", "autotune.cpp", "apply.cu", "kernels_simt.cu", "kernels_tc.cu", "hadamard_tc.cu", "pinv_tc.cu", "noalloc.cu",
           "fmm.cpp", "fmm_kernels.cu"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
PEAKS_SOURCES = ["peaks.cu"]
PEAKS_LIB = os.path.join(HERE, "libm2l_peaks.so")


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp,-O3", "-I", os.path.join(HERE, "..")] + GENCODE


def _compile(src: str) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    path = os.path.join(SRC, src)
    deps = [path] + [os.path.join(SRC, h) for h in os.listdir(SRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "m2l.h"))
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc(), "-c", path, "-o", obj] + _flags()
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _link(lib: str, objs) -> None:
    if os.path.exists(lib) and all(os.path.getmtime(lib) >= os.path.getmtime(o) for o in objs):
        return
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + list(objs) + GENCODE + ["-Xcompiler", "-fopenmp", "-lgomp", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = SOURCES + PEAKS_SOURCES
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(_compile, srcs))
    _link(LIB, objs[:len(SOURCES)])
    _link(PEAKS_LIB, objs[len(SOURCES):])
    if verbose:
        print(LIB)
        print(PEAKS_LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
