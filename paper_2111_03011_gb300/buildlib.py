"""Builds the in-tree shared library libtn_gb300.so for sm_103a.

Every translation unit is compiled in parallel; the CUDA runtime is linked
statically, so the library loads on a machine without a GPU driver (calls
that need a device then fail with TN_ERR_CUDA).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBPATH = os.path.join(LIBDIR, "libtn_gb300.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["capi.cu", "kernels.cu", "gemm_tc.cu", "noalloc.cu", "server.cu"]
CPP_SOURCES = ["planner.cpp"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _objs():
    out = []
    for s in CU_SOURCES + CPP_SOURCES:
        out.append(os.path.join(OBJDIR, os.path.splitext(s)[0] + ".o"))
    return out


def _stale():
    if not os.path.exists(LIBPATH):
        return True
    t = os.path.getmtime(LIBPATH)
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and not _stale():
        return LIBPATH
    os.makedirs(OBJDIR, exist_ok=True)
    # one builder at a time across processes (e.g. test workers importing the
    # package together); a waiter finds the library fresh and returns
    import fcntl
    with open(os.path.join(LIBDIR, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and not _stale():
            return LIBPATH
        return _build_locked(verbose, ptxas_verbose)


def _build_locked(verbose: bool, ptxas_verbose: bool) -> str:
    nvcc = _nvcc()
    jobs = []
    for s in CU_SOURCES:
        o = os.path.join(OBJDIR, os.path.splitext(s)[0] + ".o")
        cmd = [nvcc, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
               "-c", os.path.join(CSRC, s), "-o", o]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
    for s in CPP_SOURCES:
        o = os.path.join(OBJDIR, os.path.splitext(s)[0] + ".o")
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-pthread", "-I", INCLUDE,
                     "-I", os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include"),
                     "-c", os.path.join(CSRC, s), "-o", o])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    tmp = LIBPATH + ".tmp"
    link = [nvcc, "-shared", *ARCH, "-cudart", "static", "-Xcompiler", "-pthread", "-o", tmp, *_objs()]
    logs.append(_run(link))
    os.replace(tmp, LIBPATH)          # a concurrent loader never sees a partial file
    if verbose:
        for l in logs:
            if l.strip():
                sys.stdout.write(l)
    return LIBPATH


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv)
    print(LIBPATH)
