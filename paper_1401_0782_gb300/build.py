"""Compile the C-ABI CUDA library for sm_103a, in-tree.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``paper_1401_0782_gb300/lib/librsnegf.so``.  Rebuilds are skipped
when every object is newer than its sources.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
BUILDDIR = os.path.join(LIBDIR, "_build")
LIBNAME = "librsnegf.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "rsnegf.h"))
    return hs


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{p.stderr}")
    return p.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Build (if needed) and return the path of the shared library."""
    nvcc = nvcc_path()
    os.makedirs(BUILDDIR, exist_ok=True)
    srcs = sources()
    hdr_mtime = max(os.path.getmtime(h) for h in headers())
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILDDIR, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_mtime):
            todo.append((s, o))
    extra = []
    if os.environ.get("RSN_PTXAS_VERBOSE"):
        extra += ["-Xptxas", "-v"]
    jobs = jobs or min(len(todo) or 1, os.cpu_count() or 4)
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = {ex.submit(_compile, nvcc, s, o, extra): s for s, o in todo}
            for f in cf.as_completed(futs):
                logs.append((futs[f], f.result()))
    lib = lib_path()
    if todo or not os.path.exists(lib):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stderr}")
        os.replace(tmp, lib)
    if verbose:
        for s, log in logs:
            if log.strip():
                print(f"--- {os.path.basename(s)}\n{log}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
