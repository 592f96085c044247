"""Build libatlasgb.so in-tree (nvcc for sm_103a + g++ for the host geometry).

The translation units compile in parallel into ``_build/`` and link
into ``paper_1908_07038_gb300/libatlasgb.so``.  Host geometry is compiled
with ``-ffp-contract=off`` so that its FP64 arithmetic is evaluated exactly
as written on every host (x86-64 and aarch64 alike).

``build(boundscheck=True)`` makes the debugging variant
``libatlasgb_boundscheck.so`` (objects in ``_build_boundscheck/``): the
kernels compiled with ``-DATLASGB_BOUNDSCHECK`` check every table index
against their buffers and the calls report a violation as ATLAS_EBOUNDS.
The package loads it instead of the normal library when the environment
variable ATLASGB_BOUNDSCHECK is 1.
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libatlasgb.so")
LIB_BOUNDSCHECK = os.path.join(PKG, "libatlasgb_boundscheck.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    return [os.path.join(CSRC, f) for f in ("geometry.cpp", "remap.cpp", "regional.cpp", "geomio.cpp", "capi.cpp", "kernels.cu", "group.cu", "group_f32.cu", "group_bf16.cu", "noalloc.cu")]


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(INCLUDE, "atlas_gb.h")]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _sources() + _headers() + [__file__])


def _compile(src: str, cuda: str, build_dir: str, defines: list) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if src.endswith(".cu"):
        cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", *ARCH, "-lineinfo",
               "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, *defines]
    else:
        cmd = ["g++", "-c", src, "-o", obj, "-O2", "-std=c++17", "-fPIC", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas",
               "-I", INCLUDE, "-I", CSRC, "-I", os.path.join(cuda, "include")]
    subprocess.check_call(cmd)
    return obj


def build(force: bool = False, verbose: bool = False, boundscheck: bool = False) -> str:
    """Compile (if sources changed) and return the path of libatlasgb.so
    (with boundscheck, of the bounds-checked variant)."""
    lib = LIB_BOUNDSCHECK if boundscheck else LIB
    if not force and not _stale(lib):
        return lib
    cuda = _cuda_home()
    build_dir = BUILD + "_boundscheck" if boundscheck else BUILD
    defines = ["-DATLASGB_BOUNDSCHECK"] if boundscheck else []
    os.makedirs(build_dir, exist_ok=True)
    with ThreadPoolExecutor(max_workers=max(4, min(8, os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, cuda, build_dir, defines), _sources()))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [os.path.join(cuda, "bin", "nvcc"), "-shared", "-o", tmp, *objs, *ARCH,
           "-Xcompiler", "-fopenmp", "-lgomp", "-Xlinker", "--no-undefined"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, boundscheck="--boundscheck" in sys.argv))
