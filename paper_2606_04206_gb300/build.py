"""Build libdlo.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each CUDA translation unit is compiled in parallel, then linked into
``paper_2606_04206_gb300/_lib/libdlo.so``.  No CMake, no torch extension machinery.

``build(debug_bounds=True)`` builds the same sources with ``-DDLO_DEBUG_BOUNDS`` into
``_lib_debug/libdlo.so``: every index the kernels take from data (candidate pairs, kinematic
kinds, work-queue items, recorded pair counts) is checked before use, a failed check sets
status bit 8 of its rod and skips the access, and the next synchronising call returns
DLO_ERR_BOUNDS.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libdlo.so")
LIBDIR_DEBUG = os.path.join(PKG, "_lib_debug")
LIB_DEBUG = os.path.join(LIBDIR_DEBUG, "libdlo.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


# Single-precision division and square root as the hardware's approximations (at most 2 ulp),
# without the IEEE-rounded versions' correction steps and slow-path branches; the elastic
# and contact kernels take several dozen of each per vertex and substep.  The transcendental
# functions keep their accurate versions.
FAST_DIV_SQRT = ["-prec-div=false", "-prec-sqrt=false"]


def flags(extra=()):
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            *FAST_DIV_SQRT, "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = src_list + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + [os.path.join(ROOT, "include", "dlo.h")]
    return any(os.path.getmtime(s) > t for s in deps)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False, debug_bounds: bool = False) -> str:
    """Compile every .cu under csrc/ and link libdlo.so (or the bounds-checking debug library);
    returns its path."""
    libdir, lib = (LIBDIR_DEBUG, LIB_DEBUG) if debug_bounds else (LIBDIR, LIB)
    os.makedirs(libdir, exist_ok=True)
    srcs = sources()
    if not force and not ptxas_info and not _newer(srcs, lib):
        return lib
    cc = nvcc()
    objs = []
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DDLO_DEBUG_BOUNDS"] if debug_bounds else [])

    def one(src):
        obj = os.path.join(libdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *flags(extra), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        for obj, log in ex.map(one, srcs):
            objs.append(obj)
            if verbose or ptxas_info:
                sys.stderr.write(log)
    cmd = [cc, ARCH, "-shared", "-o", lib, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv))
