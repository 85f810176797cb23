"""CPU oracle for direction-optimized BFS over a degree-separated graph.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
CPU-baseline leg of the benchmark are the only callers.  The GPU product path
never imports this module, and this module imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C, single-threaded); this file only
compiles it and marshals numpy arrays.  Every function states the passage of
Pan, Pearce, Owens, "Scalable Breadth-First Search on a GPU Cluster"
(arXiv 1803.03922) that it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ORC_ERR_INVALID = -1
ORC_ERR_OOM = -2
ORC_ERR_OVERFLOW = -3


def build(src: str = _SRC, out: str = _LIB_PATH, extra_flags=()) -> str:
    """Compile ``oracle.c`` with gcc (-O2, single-threaded) into a shared library."""
    if os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))) and not extra_flags:
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-I", _HERE, "-o", tmp, src, *extra_flags]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.orc_graph_build.restype = P
    lib.orc_graph_build.argtypes = [i32, i64, P, P]
    lib.orc_graph_free.restype = None
    lib.orc_graph_free.argtypes = [P]
    lib.orc_graph_n.restype = i32
    lib.orc_graph_n.argtypes = [P]
    lib.orc_graph_nnz.restype = i64
    lib.orc_graph_nnz.argtypes = [P]
    lib.orc_graph_copy.restype = None
    lib.orc_graph_copy.argtypes = [P, P, P]
    lib.orc_bfs.restype = ctypes.c_int
    lib.orc_bfs.argtypes = [P, i32, P, P]
    lib.orc_bfs_batch_u8.restype = ctypes.c_int
    lib.orc_bfs_batch_u8.argtypes = [P, i32, P, P, P]
    lib.orc_component_edges.restype = i64
    lib.orc_component_edges.argtypes = [P, P]
    lib.orc_validate.restype = ctypes.c_int
    lib.orc_validate.argtypes = [P, i32, P, P]
    lib.orc_separate.restype = None
    lib.orc_separate.argtypes = [P, i64, P, P, P, P]
    lib.orc_subgraph_counts.restype = None
    lib.orc_subgraph_counts.argtypes = [P, i64, P]
    lib.orc_level_counters.restype = ctypes.c_int
    lib.orc_level_counters.argtypes = [P, i32, P, i64, i32, P, P]
    lib.orc_directions.restype = ctypes.c_int
    lib.orc_directions.argtypes = [P, i32, P, i32, i64, i64, ctypes.c_double, ctypes.c_double, i32, P]
    if hasattr(lib, "orc_subgraph_directions"):
        lib.orc_subgraph_directions.restype = ctypes.c_int
        lib.orc_subgraph_directions.argtypes = [P, i32, P, i64, P, P, i32, P]
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library.  ``path`` selects
    another build of the same source, e.g. a deliberately broken copy in a test."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Graph:
    """Symmetric simple graph in caller ids (Sec. II-B; Sec. VI-A.3 edge doubling):
    self-loops dropped, both directions stored, each row ascending and unique."""

    def __init__(self, n: int, src, dst, lib=None):
        self._lib = lib or load()
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if src.shape != dst.shape:
            raise ValueError("src and dst differ in length")
        h = self._lib.orc_graph_build(int(n), int(src.size), _ptr(src), _ptr(dst))
        if not h:
            raise ValueError("oracle rejected the edge list (bad n, id out of range, or out of memory)")
        self._h = ctypes.c_void_p(h)
        self.n = int(n)
        self.nnz = int(self._lib.orc_graph_nnz(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def csr(self):
        off = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.nnz, 1), dtype=np.int32)
        self._lib.orc_graph_copy(self._h, _ptr(off), _ptr(col))
        return off, col[: self.nnz]

    def degree(self):
        off = np.empty(self.n + 1, dtype=np.int64)
        self._lib.orc_graph_copy(self._h, _ptr(off), None)
        return np.diff(off)

    def bfs(self, s: int):
        """(depth, parent): FIFO-queue hop distance and canonical parent (Sec. VI-A.3)."""
        depth = np.empty(self.n, dtype=np.int32)
        parent = np.empty(self.n, dtype=np.int32)
        rc = self._lib.orc_bfs(self._h, int(s), _ptr(depth), _ptr(parent))
        if rc:
            raise ValueError("orc_bfs failed with code %d" % rc)
        return depth, parent

    def bfs_batch_u8(self, sources):
        """uint8 depth [k, n] (255 = unreached) and int32 parent [k, n]; raises
        OverflowError when a depth exceeds 254."""
        sources = np.ascontiguousarray(sources, dtype=np.int32)
        k = sources.size
        depth = np.empty((k, self.n), dtype=np.uint8)
        parent = np.empty((k, self.n), dtype=np.int32)
        rc = self._lib.orc_bfs_batch_u8(self._h, k, _ptr(sources), _ptr(depth), _ptr(parent))
        if rc == ORC_ERR_OVERFLOW:
            raise OverflowError("a depth exceeds 254")
        if rc:
            raise ValueError("orc_bfs_batch_u8 failed with code %d" % rc)
        return depth, parent

    def component_edges(self, depth) -> int:
        depth = np.ascontiguousarray(depth, dtype=np.int32)
        return int(self._lib.orc_component_edges(self._h, _ptr(depth)))

    def validate(self, s: int, depth, parent) -> int:
        depth = np.ascontiguousarray(depth, dtype=np.int32)
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        return int(self._lib.orc_validate(self._h, int(s), _ptr(depth), _ptr(parent)))

    def separate(self, th: int):
        """Degree separation (Sec. III-A, Fig. 2): returns (internal_of, caller_of, d, n_ni)."""
        internal_of = np.empty(self.n, dtype=np.int32)
        caller_of = np.empty(self.n, dtype=np.int32)
        d = ctypes.c_int32()
        n_ni = ctypes.c_int32()
        self._lib.orc_separate(self._h, int(th), _ptr(internal_of), _ptr(caller_of),
                               ctypes.byref(d), ctypes.byref(n_ni))
        return internal_of, caller_of, int(d.value), int(n_ni.value)

    def level_counters(self, s: int, depth, th: int, dirs):
        """Per-level work counters [levels, 7] for the given directions (see oracle.h)."""
        depth = np.ascontiguousarray(depth, dtype=np.int32)
        dirs = np.ascontiguousarray(dirs, dtype=np.int32)
        out = np.zeros((dirs.size, 7), dtype=np.int64)
        rc = self._lib.orc_level_counters(self._h, int(s), _ptr(depth), int(th), dirs.size, _ptr(dirs), _ptr(out))
        if rc:
            raise ValueError("orc_level_counters failed with code %d" % rc)
        return out

    def directions(self, s: int, depth, rule: str = "beamer", alpha: int = 15, beta: int = 18,
                   factor0: float = 0.5, factor1: float = 1e-7):
        """Per-level directions (0 forward, 1 backward) that the rule ("beamer",
        "beamer_stay" or "paper", Sec. IV-B) takes on the run from s with final depth `depth`."""
        depth = np.ascontiguousarray(depth, dtype=np.int32)
        cap = int(depth.max()) + 2 if depth.size else 1
        out = np.zeros(cap, dtype=np.int32)
        code = {"beamer": 0, "paper": 1, "beamer_stay": 2}[rule]
        rc = self._lib.orc_directions(self._h, int(s), _ptr(depth), code, int(alpha), int(beta), float(factor0),
                                      float(factor1), cap, _ptr(out))
        if rc < 0:
            raise ValueError("orc_directions failed with code %d" % rc)
        return out[:rc].copy()

    def subgraph_directions(self, s: int, depth, th: int, factor0=(0.5, 0.05, 1e-7), factor1=(1e-7, 1e-7, 1e-7)):
        """Per-level directions of the dd, dn and nd visits (Sec. IV-B, each with its
        own factor pair; nn always forward) on the run from s: int32 [levels],
        bit 0 dd, bit 1 dn, bit 2 nd backward."""
        depth = np.ascontiguousarray(depth, dtype=np.int32)
        cap = int(depth.max()) + 2 if depth.size else 1
        out = np.zeros(cap, dtype=np.int32)
        f0 = np.ascontiguousarray(factor0, dtype=np.float64)
        f1 = np.ascontiguousarray(factor1, dtype=np.float64)
        rc = self._lib.orc_subgraph_directions(self._h, int(s), _ptr(depth), int(th), _ptr(f0), _ptr(f1), cap,
                                               _ptr(out))
        if rc < 0:
            raise ValueError("orc_subgraph_directions failed with code %d" % rc)
        return out[:rc].copy()

    def subgraph_counts(self, th: int):
        """Directed entry counts (|E_nn|, |E_nd|, |E_dn|, |E_dd|) for threshold th (Sec. IV)."""
        out = np.zeros(4, dtype=np.int64)
        self._lib.orc_subgraph_counts(self._h, int(th), _ptr(out))
        return out
