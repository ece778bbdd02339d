"""Build libndsi.so (host analysis + sm_103a kernels + C ABI) in-tree with nvcc and g++."""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build", platform.machine())
LIB = os.path.join(PKG, "libndsi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels.cu", "api.cu", "api_mu.cu", "api_solve.cu", "static_scratch.cu", "split_gemm.cu", "mlp.cu",
              "solve.cu", "peak.cu"]
CPP_SOURCES = ["analyze.cpp", "mu_search.cpp", "plan_check.cpp", "small_eig.cpp"]
HEADERS = ["plan.hpp", "kernels.cuh", "split_gemm.cuh", "solve.cuh", "handle.hpp", "small_eig.hpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libndsi.so")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stderr


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every translation unit (in parallel) and link the shared library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "ndsi.h")]
    jobs, objs = [], []
    common = ["-O3", "-std=c++17", "-I" + INCLUDE, "-I" + CSRC]
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc] + ARCH + common + ["-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"
                                                  if verbose else "-O3", "-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append(["g++"] + common + ["-fPIC", "-Wall", "-c", s, "-o", o])
    if jobs:
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            for log in ex.map(_compile, jobs):
                if verbose and log:
                    sys.stderr.write(log)
    if force or jobs or _stale(LIB, objs):
        _compile([nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart_static", "-lrt", "-ldl",
                                                                  "-lpthread"])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
