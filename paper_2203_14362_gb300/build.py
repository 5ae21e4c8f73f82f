"""Build libspx.so in-tree for sm_103a (nvcc for the CUDA sources, g++ for the
host index build), compiling translation units in parallel."""
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
LIB = os.path.join(PKG, "libspx.so")
# the debug flavour: every index walk of the kernels bounds-checked (SPX_BOUNDS_CHECK)
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libspx_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels.cu", "api.cu", "server.cu", "index_build_device.cu"]
CPP_SOURCES = ["index_build.cpp", "disk_index.cpp", "buffer_index.cpp"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libspx")


def _run(cmd: list[str], verbose: bool) -> None:
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}")
    if verbose and r.stdout.strip():
        print(r.stdout, flush=True)


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "spx.h"), __file__]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, checked: bool = False) -> str:
    """Compile and link libspx.so next to this file (checked: the
    bounds-checked debug flavour, libspx_checked.so); returns its path."""
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    if not force and not _stale(lib):
        return lib
    nv = nvcc()
    # SPX_NVCC_EXTRA: extra nvcc flags, e.g. -D settings of the kernels' tuning macros
    common = ["-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE] + (["-DSPX_BOUNDS_CHECK"] if checked else [])
    extra = os.environ.get("SPX_NVCC_EXTRA", "").split()
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(build_dir, f + ".o")
        objs.append(o)
        cmd = [nv, *ARCH, "-lineinfo", *common, *extra, "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
               "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
    for f in CPP_SOURCES:
        o = os.path.join(build_dir, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-I", CSRC, "-I", INCLUDE,
                     "-c", os.path.join(CSRC, f), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for fut in [ex.submit(_run, j, verbose) for j in jobs]:
            fut.result()
    tmp = lib + f".{os.getpid()}.tmp"
    _run([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], verbose)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
