"""Build the CUDA library libsimplexgb.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into
paper_0912_4273_gb300/_build/libsimplexgb.so.  No cmake, no torch extension
machinery: the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")  # -DSX_DEBUG: the kernels check their indices
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBNAME = "libsimplexgb.so"
SOURCES = ["sx_api.cu", "sx_setup.cu", "sx_step.cu", "sx_ballistic.cu", "sx_update.cu", "sx_halo.cu",
           "sx_noalloc.cu", "sx_remesh.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def lib_path(debug: bool = False) -> str:
    return os.path.join(BUILD_DEBUG if debug else BUILD, LIBNAME)


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile the library (with debug, a second build with -DSX_DEBUG into
    its own folder); returns its path."""
    bdir = BUILD_DEBUG if debug else BUILD
    if debug:
        extra = ["-DSX_DEBUG", *extra]
    os.makedirs(bdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    objs = []
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(bdir, os.path.splitext(s)[0] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, __file__] + headers):
            jobs.append([nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
            if verbose and (r.stdout or r.stderr):
                print(r.stdout + r.stderr)
    out = lib_path(debug)
    if force or jobs or _stale(out, objs):
        tmp = out + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
