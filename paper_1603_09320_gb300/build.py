"""Compiles the C-ABI library libhnsw_gb300.so in-tree (sm_103a only).

    python -m paper_1603_09320_gb300.build [--verbose]

Translation units are compiled in parallel, then linked with nvcc.  The
result is paper_1603_09320_gb300/_build/libhnsw_gb300.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhnsw_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", INCLUDE]
CXX_FLAGS = ["-O3", "-std=c++17", "-fPIC", "-pthread", "-I", INCLUDE, "-I", "/usr/local/cuda/include"]

SOURCES = ["search.cu", "search_noalloc.cu", "merge.cu", "index.cu", "stopnet.cu", "gpu_build.cu", "builder.cpp", "blob.cpp",
           "server.cpp"]
HEADERS = ["common.hpp", "index.cuh", "stopnet.cuh"]


def _obj(src: str) -> str:
    return os.path.join(BUILD, src + ".o")


def _compile(src: str, verbose: bool) -> str:
    path = os.path.join(CSRC, src)
    out = _obj(src)
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, *CU_FLAGS, "-c", path, "-o", out]
        if verbose:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd = ["g++", *CXX_FLAGS, "-c", path, "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stderr if verbose else ""


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "hnsw.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale():
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if verbose:
        for lg in logs:
            if lg:
                print(lg, file=sys.stderr)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *[_obj(s) for s in SOURCES], "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv))
