"""Build ``libsorgb.so`` (the C-ABI library of include/sor.h) for sm_103a.

nvcc compiles each translation unit in parallel and links a shared library
into ``paper_1401_0763_gb300/_build/``.  No CMake, no torch extension
machinery: the library has a plain C ABI and is loaded with ctypes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libsorgb.so")
# debug variant: device-side index checks (SOR_DEBUG_BOUNDS) that turn an
# access outside a slot's arrays into a solve error instead of a fault
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libsorgb.so")
SOURCES = ["sor_kernels.cu", "sor_cluster.cu", "sor_runtime.cu", "sor_batch.cu", "sor_capi.cu", "sor_static.cu",
           "sor3d.cu", "sor9.cu", "sor_probe.cu", "sor_wf.cu", "sor_tile.cu", "sor_grid.cu", "sor_block.cu"]
HEADERS = ["sor_device.cuh", "sor_devfn.cuh", "sor_bits.cuh", "sor_strips.cuh", "sor_kernels.h", "sor_runtime.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsorgb.so")


def _stamp() -> float:
    paths = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    paths += [os.path.join(ROOT, "include", "sor.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link; returns the library path.  Skips work when the
    library is newer than every source.  debug=True builds the variant with
    device-side index checks into its own directory."""
    build_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _stamp():
        return lib
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    objs = []
    extra = ["-DSOR_DEBUG_BOUNDS"] if debug else []

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
