"""Build libxyl.so in-tree for sm_103a (nvcc + g++, no cmake).

Each translation unit compiles in its own process, in parallel; the shared
library links the CUDA runtime dynamically so that it shares the runtime torch
already loaded.  build(debug=True) makes libxyl_debug.so instead: the same
sources compiled with XYL_DEBUG, whose kernels check every neighbour id, row
length and colour-class bound before following it (a bad one sets the status
word to XYL_EBOUNDS and is skipped); the binding loads it when the
environment sets XYL_DEBUG=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libxyl.so")
LIB_DEBUG = os.path.join(HERE, "libxyl_debug.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
CU_SOURCES = ["common.cu", "plain.cu", "batched.cu", "resident.cu", "resident_o3.cu", "plan.cu", "walk.cu", "o3.cu"]
CXX_SOURCES = ["graph.cpp"]
# FP64 engine and spin initialisation: every expression evaluated as written (no
# FMA contraction), so their arithmetic is a fixed sequence of IEEE operations
NO_FMA_SOURCES = {"common.cu", "plain.cu", "o3.cu"}


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stdout + res.stderr


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(HERE, "..", "include", "xyl.h")]


def needs_build(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile every translation unit and link libxyl.so (libxyl_debug.so with
    debug=True); returns its path."""
    lib = LIB_DEBUG if debug else LIB
    if not force and not needs_build(debug):
        return lib
    build_dir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include")]
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(build_dir, f + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
               "-c", os.path.join(CSRC, f), "-o", obj] + inc
        if debug:
            cmd.insert(2, "-DXYL_DEBUG")
        if f in NO_FMA_SOURCES:
            cmd.insert(2, "-fmad=false")
        if ptxas_info:
            cmd.insert(2, "-Xptxas=-v")
        jobs.append((obj, cmd))
    for f in CXX_SOURCES:
        obj = os.path.join(build_dir, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
               "-I", "/usr/local/cuda/include", "-c", os.path.join(CSRC, f), "-o", obj] + inc
        jobs.append((obj, cmd))
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[1]), jobs))
    if verbose or ptxas_info:
        for o in outs:
            if o.strip():
                print(o)
    tmp = lib + f".tmp{os.getpid()}"
    _run([nvcc, ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64", "-o", tmp]
         + [j[0] for j in jobs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, ptxas_info="-v" in sys.argv, debug="--debug" in sys.argv))
