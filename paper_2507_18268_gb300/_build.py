"""Builds liblapfoam.so (the CUDA path) in-tree for sm_103a with nvcc.

Each .cu translation unit compiles in parallel to an object file under ``_lib/obj``; the
objects link into ``_lib/liblapfoam.so``. A rebuild happens when any source or header is
newer than the library. ``checked=True`` builds the checked variant (``-DLFM_CHECKED``:
every index a kernel reads from the mesh addressing is tested before use) into
``_lib/liblapfoam_checked.so`` from objects under ``_lib/obj_checked``.
"""
from __future__ import annotations

import concurrent.futures
import fcntl
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblapfoam.so")
CHECKED_LIB = os.path.join(LIBDIR, "liblapfoam_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def lib_path(checked: bool = False) -> str:
    return CHECKED_LIB if checked else LIB


def up_to_date(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles the CUDA sources (if stale) and returns the library path."""
    lib = lib_path(checked)
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else "obj")
    flags = NVCC_FLAGS + (["-DLFM_CHECKED"] if checked else [])
    os.makedirs(objdir, exist_ok=True)
    with open(os.path.join(LIBDIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if not force and up_to_date(checked):
            return lib
        nvcc = _nvcc()

        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc] + flags + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout + r.stderr)
            return obj

        with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(sources()))) as ex:
            objs = list(ex.map(compile_one, sources()))
        tmp = lib + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
        return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
