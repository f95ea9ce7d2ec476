"""Build libplbm.so (sm_103a) in-tree with nvcc.

Every CUDA and host translation unit under ``csrc/`` is compiled in parallel
with ``-gencode arch=compute_103a,code=sm_103a`` and linked into
``_build/libplbm.so`` next to this file.  No CMake, no setuptools.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libplbm.so")

SOURCES = [
    "plbm_host.cpp",
    "plbm_stability.cpp",
    "plbm_aux.cu",
    "plbm_step_f64.cu",
    "plbm_step_f32.cu",
    "plbm_step_f16.cu",
    "plbm_step3.cu",
    "plbm_step_bf16.cu",
    "plbm_noalloc.cu",
    "plbm_slabs.cu",
    "plbm_cnn.cu",
    "plbm_cnn_tc.cu",
    "plbm_ce.cu",
    "plbm_surrogate.cpp",
]
HEADERS = ["plbm_internal.h", "plbm_device.cuh", "plbm_pair.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libplbm")
    return exe


def _flags(verbose_ptxas: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _newest_input() -> float:
    paths = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "plbm.h"),
                                                                   os.path.abspath(__file__)]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose_ptxas: bool | None = None) -> str:
    """Compile and link libplbm.so; returns its path.  Skips work when up to date."""
    if verbose_ptxas is None:
        verbose_ptxas = os.environ.get("PLBM_PTXAS_VERBOSE", "") == "1"
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    flags = _flags(verbose_ptxas)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [exe] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
