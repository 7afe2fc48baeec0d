"""Compile libmsgs.so (the CUDA library behind include/msgs.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library next to this file.  No fast-math: the footprint stage
relies on IEEE single-precision rounding.  build(debug=True) makes
libmsgs_debug.so, the same sources compiled with -DMS_DEBUG: index checks
in the kernels that report through the status word (MS_ERR_BOUNDS), for
the tests; the binding loads it when MSGS_DEBUG=1.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmsgs.so")
LIB_DEBUG = os.path.join(HERE, "libmsgs_debug.so")
SOURCES = ["api.cu", "project.cu", "bin.cu", "raster.cu", "raster_list.cu", "raster_group.cu", "backward.cu",
           "serve.cu", "aggregate.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-Wall", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _nvcc_path(nvcc):
    import shutil
    return nvcc if os.path.sep in nvcc else (shutil.which(nvcc) or nvcc)


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(debug):
        return lib
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    flags = list(extra_flags) + (["-DMS_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    home = os.path.dirname(os.path.dirname(_nvcc_path(nvcc)))
    rpaths = sorted({os.path.join(home, "lib64"),
                     os.path.join(os.path.realpath(home), "lib64")})
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared",
           "-Xlinker", "-rpath," + ":".join(rpaths), "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
