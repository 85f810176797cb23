"""Compiles the CUDA sources of the package into an in-tree shared library for
sm_103a (nvcc, one -gencode, translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbfs_gb300.so")
# the bounds-checked build (-DBFS_CHECK): an index outside its array sets
# BFS_ERR_CHECK in the run's status instead of being accessed
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(PKG, "libbfs_gb300_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest(extra=()):
    h = hashlib.sha256()
    files = sources() + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    files.append(os.path.join(INCLUDE, "bfs_gb300.h"))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compiles the library (check=True: the bounds-checked build) and returns its path."""
    bdir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    extra = ["-DBFS_CHECK"] if check else []
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "stamp")
    dig = _digest(extra)
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == dig:
        return lib

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = ["nvcc", *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        with open(obj + ".ptxas.txt", "w") as fh:
            fh.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    with open(stamp, "w") as fh:
        fh.write(dig)
    if verbose:
        for o in objs:
            print(open(o + ".ptxas.txt").read())
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
