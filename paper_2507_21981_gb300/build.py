"""Builds libdgs.so in-tree for sm_103a (nvcc, one -gencode, translation units in parallel), and
libdgs_debug.so, the same sources compiled with -DDGS_DEBUG (device bounds checks on every index
a kernel takes from another kernel's output; see dgs_build_flags in include/dgs.h)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgs.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libdgs_debug.so")
SOURCES = ["api.cu", "project.cu", "sort.cu", "binning.cu", "composite.cu", "backward.cu", "noalloc.cu", "layout.cu",
           "augment.cu", "lidar.cu", "mesh.cu", "tsdf.cu"]
HEADERS = [os.path.join(CSRC, "dgs_internal.cuh"), os.path.join(INCLUDE, "dgs.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdgs")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds libdgs.so (or, with debug, libdgs_debug.so) if any source is newer; returns its path."""
    out_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    flags = FLAGS + (["-DDGS_DEBUG"] if debug else [])
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out_dir, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + HEADERS):
            jobs.append([cc, *ARCH, *flags, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode:
                print(" ".join(cmd)); print(r.stdout); print(r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode:
            print(r.stdout, r.stderr)
            raise RuntimeError(f"link of {os.path.basename(lib)} failed")
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> None:
    """Both libraries, their translation units compiled together."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(build, force, verbose, d) for d in (False, True)]:
            f.result()


if __name__ == "__main__":
    build_all(verbose=True)
    print(LIB, LIB_DEBUG)
