"""Direction-optimized BFS over a degree-separated graph on one GB300 (sm_103a).

Thin ctypes binding of the C ABI declared in ``include/bfs_gb300.h``: the
functions below carry the same names and only marshal arguments (PyTorch tensors
or numpy arrays to pointers, streams to ``cudaStream_t``).  Every step of the
BFS runs in the CUDA kernels of ``libbfs_gb300.so``; there is no other path, and
importing this package fails loudly when that library is missing.

Method: Pan, Pearce, Owens, "Scalable Breadth-First Search on a GPU Cluster"
(arXiv 1803.03922): degree separation (Sec. III-A), forward and backward visits
(Sec. IV-A/B), direction optimization (Sec. IV-B), hop distance output
(Sec. VI-A.3) plus a canonical BFS-tree parent.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

BFS_OK = 0
BFS_ERR_INVALID = -1
BFS_ERR_OOM = -2
BFS_ERR_OVERFLOW = -3
BFS_ERR_TIMEOUT = -4
BFS_ERR_CUDA = -5
BFS_ERR_CHECK = -6

BFS_SCHED_BEAMER = 0
BFS_SCHED_TOPDOWN = 1
BFS_SCHED_BOTTOMUP = 2
BFS_SCHED_ALTERNATE = 3
BFS_SCHED_MASK = 4
BFS_SCHED_PAPER = 5
BFS_SCHED_PAPER_SUBGRAPH = 6
BFS_SCHED_BEAMER_STAY = 7

BFS_TD_PARENT_PULL = 0
BFS_TD_PARENT_ATOMICMIN = 1

BFS_LOG_LEVELS = 256

c_i32, c_i64, c_u64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class bfs_options(ctypes.Structure):
    _fields_ = [("th", c_i64), ("edges_on_device", c_i32), ("schedule", c_i32), ("schedule_mask", c_u64),
                ("alpha", c_i32), ("beta", c_i32), ("factor0", c_dbl), ("factor1", c_dbl),
                ("td_parent", c_i32), ("blocks_per_sm", c_i32), ("barrier_timeout_ms", c_i32),
                ("test_skip_barrier", c_i32), ("run_timeout_ms", c_i32), ("tuning", c_i32),
                ("subgraph_factor0", c_dbl * 3), ("subgraph_factor1", c_dbl * 3), ("reserved", c_i32 * 4)]


class bfs_graph_info(ctypes.Structure):
    _fields_ = [("n", c_i32), ("n_nonisolated", c_i32), ("delegates", c_i32), ("grid_blocks", c_i32),
                ("th", c_i64), ("nnz", c_i64), ("max_degree", c_i64), ("subgraph_edges", c_i64 * 4),
                ("chunk_capacity", c_i64), ("device_bytes", c_i64)]


class bfs_level_log(ctypes.Structure):
    _fields_ = [("direction", c_i32), ("converted", c_i32), ("frontier", c_i64), ("frontier_edges", c_i64),
                ("scanned", c_i64), ("edges_examined", c_i64), ("parent_edges", c_i64), ("found", c_i64),
                ("queue_entries", c_i64), ("t_begin_ns", c_u64), ("t_expand_ns", c_u64), ("t_end_ns", c_u64),
                ("t_first_done_ns", c_u64), ("t_last_done_ns", c_u64), ("subgraph_directions", c_i32),
                ("reserved", c_i32)]


class bfs_stats(ctypes.Structure):
    _fields_ = [("levels", c_i32), ("logged_levels", c_i32), ("reached", c_i64), ("component_edges", c_i64),
                ("edges_examined", c_i64), ("model_bytes", c_i64), ("device_ns", c_u64), ("setup_ns", c_u64),
                ("result_ns", c_u64),
                ("level", bfs_level_log * BFS_LOG_LEVELS)]


BFS_BATCH_LOG_LEVELS = 64


class bfs_batch_level(ctypes.Structure):
    _fields_ = [("direction", c_i32), ("pulled_lanes", c_i32), ("frontier_vertices", c_i64), ("frontier_edges", c_i64),
                ("pairs", c_i64), ("t_begin_ns", c_u64), ("t_expand_ns", c_u64), ("t_end_ns", c_u64)]


class bfs_batch_stats(ctypes.Structure):
    _fields_ = [("levels", c_i32), ("logged_levels", c_i32), ("pairs_reached", c_i64), ("traversed_edges", c_i64),
                ("device_ns", c_u64), ("setup_ns", c_u64), ("result_ns", c_u64),
                ("level", bfs_batch_level * BFS_BATCH_LOG_LEVELS)]


class bfs_server_options(ctypes.Structure):
    _fields_ = [("max_concurrent", c_i32), ("max_lanes", c_i32), ("with_parents", c_i32),
                ("contexts_per_graph", c_i32), ("hbm_reserve_bytes", c_i64), ("hbm_budget_bytes", c_i64),
                ("single_path", c_i32), ("single_max", c_i32), ("group_batches", c_i32),
                ("reserved", c_i32 * 5)]


class bfs_server_done(ctypes.Structure):
    _fields_ = [("ticket", c_i64), ("status", c_i32), ("graph_id", c_i32), ("batch_size", c_i32),
                ("levels", c_i32), ("t_arrival_ns", c_i64), ("t_launch_ns", c_i64), ("t_done_ns", c_i64),
                ("device_ns", c_i64)]


class bfs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", c_i64), ("completed", c_i64), ("failed", c_i64), ("launches", c_i64),
                ("lanes_launched", c_i64), ("contexts_created", c_i64), ("contexts_evicted", c_i64),
                ("context_bytes", c_i64), ("waiting", c_i64), ("in_flight", c_i64),
                ("capacity_ctas", c_i32), ("ctas_per_launch", c_i32), ("single_launches", c_i64),
                ("reserved", c_i64 * 3)]


class BfsError(RuntimeError):
    def __init__(self, code, message):
        super().__init__("bfs error %d: %s" % (code, message))
        self.code = code


_lib = None


def _load():
    """The CUDA library: libbfs_gb300.so, or the build named by the environment
    variable BFS_GB300_LIB (the bounds-checked build, libbfs_gb300_check.so)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("BFS_GB300_LIB") or _build.LIB
    if not os.path.exists(path):
        raise ImportError("%s is not built; run __graft_entry__.build() "
                          "(the CUDA library is the only implementation)" % os.path.basename(path))
    lib = ctypes.CDLL(path)
    lib.bfs_options_default.argtypes = [ctypes.POINTER(bfs_options)]
    lib.bfs_build_graph.argtypes = [c_vp, c_vp, c_i64, c_i32, ctypes.POINTER(bfs_options),
                                    ctypes.POINTER(c_vp), c_vp]
    lib.bfs_set_options.argtypes = [c_vp, ctypes.POINTER(bfs_options)]
    lib.bfs_graph_get_info.argtypes = [c_vp, ctypes.POINTER(bfs_graph_info)]
    lib.bfs_graph_export.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp]
    lib.bfs_run.argtypes = [c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(bfs_stats), c_vp]
    lib.bfs_run_many.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]
    lib.bfs_wait.argtypes = [c_vp, c_vp]
    lib.bfs_run_static.argtypes = [c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp]
    lib.bfs_free.argtypes = [c_vp]
    lib.bfs_free.restype = None
    lib.bfs_last_error.restype = ctypes.c_char_p
    lib.bfs_last_error.argtypes = []
    lib.bfs_batch_create.argtypes = [c_vp, c_i32, c_i32, ctypes.POINTER(c_vp)]
    lib.bfs_batch_capacity.argtypes = [ctypes.POINTER(c_i32)]
    lib.bfs_batch_device_bytes.argtypes = [c_vp]
    lib.bfs_batch_device_bytes.restype = c_i64
    lib.bfs_run_batch.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(bfs_batch_stats), c_vp]
    lib.bfs_batch_wait.argtypes = [c_vp, c_vp]
    lib.bfs_batch_free.argtypes = [c_vp]
    lib.bfs_batch_free.restype = None
    lib.bfs_batch_order.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp]
    lib.bfs_degree_class_stats.argtypes = [c_vp, c_vp, c_i32, c_vp, c_vp]
    lib.bfs_server_options_default.argtypes = [ctypes.POINTER(bfs_server_options)]
    lib.bfs_server_options_default.restype = None
    lib.bfs_server_create.argtypes = [ctypes.POINTER(bfs_server_options), ctypes.POINTER(c_vp)]
    lib.bfs_server_add_graph.argtypes = [c_vp, c_vp, ctypes.POINTER(c_i32)]
    lib.bfs_server_now_ns.argtypes = []
    lib.bfs_server_now_ns.restype = c_i64
    lib.bfs_server_submit.argtypes = [c_vp, c_i32, c_i32, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]
    lib.bfs_server_poll.argtypes = [c_vp, ctypes.POINTER(bfs_server_done), c_i32, c_i32, ctypes.POINTER(c_i32)]
    lib.bfs_server_get_stats.argtypes = [c_vp, ctypes.POINTER(bfs_server_stats)]
    lib.bfs_server_destroy.argtypes = [c_vp]
    lib.bfs_server_destroy.restype = None
    lib.bfs_server_abi_sizes.argtypes = [ctypes.POINTER(c_i64 * 3)]
    lib.bfs_server_abi_sizes.restype = None
    ssz = (c_i64 * 3)()
    lib.bfs_server_abi_sizes(ctypes.byref(ssz))
    swant = [ctypes.sizeof(t) for t in (bfs_server_options, bfs_server_done, bfs_server_stats)]
    if list(ssz) != swant:
        raise ImportError("server ABI struct sizes differ: library %s, binding %s" % (list(ssz), swant))
    lib.bfs_abi_sizes.argtypes = [ctypes.POINTER(c_i64 * 5)]
    lib.bfs_abi_sizes.restype = None
    sizes = (c_i64 * 5)()
    lib.bfs_abi_sizes(ctypes.byref(sizes))
    want = [ctypes.sizeof(t) for t in (bfs_options, bfs_graph_info, bfs_level_log, bfs_stats, bfs_batch_stats)]
    if list(sizes) != want:
        raise ImportError("ABI struct sizes differ: library %s, binding %s" % (list(sizes), want))
    _lib = lib
    return lib


def library_path() -> str:
    return _build.LIB


def _check(rc):
    if rc != BFS_OK:
        raise BfsError(rc, bfs_last_error())
    return rc


def _ptr(x):
    """Pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return c_vp(x.ctypes.data)
    return c_vp(x.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        if not torch.cuda.is_available():
            return None
        return c_vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_vp(stream)
    return c_vp(stream.cuda_stream)


# ---- the C ABI, one function per entry point -------------------------------------------------

def bfs_last_error() -> str:
    return _load().bfs_last_error().decode()


def bfs_options_default() -> bfs_options:
    o = bfs_options()
    _check(_load().bfs_options_default(ctypes.byref(o)))
    return o


def bfs_build_graph(src, dst, num_vertices: int, opt: bfs_options | None = None, stream=None):
    """Returns an opaque handle.  src/dst: int32 CUDA tensors, or int32 host
    arrays/tensors (``opt.edges_on_device`` is set from where they live)."""
    lib = _load()
    o = opt if opt is not None else bfs_options_default()
    on_dev = not isinstance(src, np.ndarray) and getattr(src, "is_cuda", False)
    o.edges_on_device = 1 if on_dev else 0
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        m = src.size
    else:
        if src.dtype != dst.dtype or str(src.dtype) != "torch.int32" or not src.is_contiguous() or \
                not dst.is_contiguous():
            raise ValueError("src and dst must be contiguous int32")
        m = src.numel()
    if (dst.size if isinstance(dst, np.ndarray) else dst.numel()) != m:
        raise ValueError("src and dst differ in length")
    h = c_vp()
    _check(lib.bfs_build_graph(_ptr(src), _ptr(dst), m, int(num_vertices), ctypes.byref(o), ctypes.byref(h),
                               _stream(stream)))
    return h


def bfs_set_options(g, opt: bfs_options):
    _check(_load().bfs_set_options(g, ctypes.byref(opt)))


def bfs_graph_get_info(g) -> bfs_graph_info:
    info = bfs_graph_info()
    _check(_load().bfs_graph_get_info(g, ctypes.byref(info)))
    return info


def bfs_graph_export(g):
    """(row_off, col, caller_of, internal_of) as numpy arrays (internal ids)."""
    info = bfs_graph_get_info(g)
    off = np.empty(info.n_nonisolated + 1, dtype=np.int64)
    col = np.empty(max(info.nnz, 1), dtype=np.int32)
    co = np.empty(info.n, dtype=np.int32)
    io = np.empty(info.n, dtype=np.int32)
    _check(_load().bfs_graph_export(g, _ptr(off), _ptr(col), _ptr(co), _ptr(io)))
    return off, col[: info.nnz], co, io


def bfs_run(g, source: int, depth, parent, stats: bfs_stats | None = None, stream=None):
    """depth/parent: int32 buffers of n entries, both CUDA tensors or both host
    (numpy arrays / pinned tensors)."""
    _check(_load().bfs_run(g, int(source), _ptr(depth), _ptr(parent),
                           ctypes.byref(stats) if stats is not None else None, _stream(stream)))


def bfs_run_many(g, sources, depth, parent, status=None, stream=None):
    """Pipelined runs with host results: sources (ints), depth/parent: lists of
    host int32 buffers (numpy arrays / pinned tensors) of n entries, one pair per
    source; status: optional int32 numpy array of len(sources)."""
    k = len(sources)
    if len(depth) != k or len(parent) != k:
        raise ValueError("one depth and one parent buffer per source")
    src = (c_i32 * max(k, 1))(*[int(x) for x in sources])
    dp = (c_vp * max(k, 1))(*[_ptr(x).value for x in depth])
    pp = (c_vp * max(k, 1))(*[_ptr(x).value for x in parent])
    st = None
    if status is not None:
        if not (isinstance(status, np.ndarray) and status.dtype == np.int32 and status.size >= k):
            raise ValueError("status must be an int32 numpy array of len(sources)")
        st = c_vp(status.ctypes.data)
    _check(_load().bfs_run_many(g, src, int(k), dp, pp, st, _stream(stream)))


def bfs_wait(g, stream=None):
    _check(_load().bfs_wait(g, _stream(stream)))


def bfs_run_static(row_off, col, n: int, source: int, depth, parent, stream=None):
    """The allocation-free entry point: caller-owned device CSR (int64 offsets,
    int32 sorted symmetric columns) and device result buffers."""
    _check(_load().bfs_run_static(_ptr(row_off), _ptr(col), int(n), int(source), _ptr(depth), _ptr(parent),
                                  _stream(stream)))


def bfs_batch_create(g, with_parents: bool = True, ctas: int = 0):
    h = c_vp()
    _check(_load().bfs_batch_create(g, 1 if with_parents else 0, int(ctas), ctypes.byref(h)))
    return h


def bfs_batch_capacity() -> int:
    c = c_i32()
    _check(_load().bfs_batch_capacity(ctypes.byref(c)))
    return int(c.value)


def bfs_batch_device_bytes(b) -> int:
    return int(_load().bfs_batch_device_bytes(b))


def bfs_run_batch(b, sources, depth, parent=None, stats: bfs_batch_stats | None = None, stream=None):
    """sources: host int32 array (1..64 caller ids); depth uint8 [k*n], parent int32 [k*n]
    (or None), both device tensors or both host arrays/pinned tensors."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    _check(_load().bfs_run_batch(b, _ptr(src), src.size, _ptr(depth), _ptr(parent),
                                 ctypes.byref(stats) if stats is not None else None, _stream(stream)))


def bfs_batch_wait(b, stream=None):
    _check(_load().bfs_batch_wait(b, _stream(stream)))


def bfs_batch_free(b):
    if b:
        _load().bfs_batch_free(b)


def bfs_batch_order(g, sources, stream=None):
    """Permutation (int32 numpy array) grouping the sources for batching: by the
    degree sum of each source's neighbours, largest first."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    order = np.empty(src.size, dtype=np.int32)
    _check(_load().bfs_batch_order(g, _ptr(src), src.size, _ptr(order), _stream(stream)))
    return order


def bfs_degree_class_stats(g, ths, stream=None):
    """[len(ths), 5] int64: delegates, |E_nn|, |E_nd|, |E_dn|, |E_dd| per threshold."""
    t = np.ascontiguousarray(ths, dtype=np.int64)
    out = np.zeros((t.size, 5), dtype=np.int64)
    _check(_load().bfs_degree_class_stats(g, _ptr(t), t.size, _ptr(out), _stream(stream)))
    return out


def bfs_server_options_default() -> bfs_server_options:
    o = bfs_server_options()
    _load().bfs_server_options_default(ctypes.byref(o))
    return o


def bfs_server_create(opt: bfs_server_options | None = None):
    h = c_vp()
    _check(_load().bfs_server_create(ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def bfs_server_add_graph(s, g) -> int:
    gid = c_i32()
    _check(_load().bfs_server_add_graph(s, g, ctypes.byref(gid)))
    return int(gid.value)


def bfs_server_now_ns() -> int:
    return int(_load().bfs_server_now_ns())


def bfs_server_submit(s, graph_id: int, source: int, depth, parent=None, t_arrival_ns: int = 0) -> int:
    t = c_i64()
    _check(_load().bfs_server_submit(s, int(graph_id), int(source), _ptr(depth), _ptr(parent),
                                     int(t_arrival_ns), ctypes.byref(t)))
    return int(t.value)


def bfs_server_poll(s, max_done: int = 256, timeout_ms: int = 0):
    buf = (bfs_server_done * max_done)()
    n = c_i32()
    _check(_load().bfs_server_poll(s, buf, int(max_done), int(timeout_ms), ctypes.byref(n)))
    return [buf[i] for i in range(n.value)]


def bfs_server_get_stats(s) -> bfs_server_stats:
    st = bfs_server_stats()
    _check(_load().bfs_server_get_stats(s, ctypes.byref(st)))
    return st


def bfs_server_destroy(s):
    if s:
        _load().bfs_server_destroy(s)


def bfs_free(g):
    if g:
        _load().bfs_free(g)


# ---- convenience wrapper ---------------------------------------------------------------------

class Graph:
    """A device-resident degree-separated graph and its BFS runs."""

    def __init__(self, src, dst, num_vertices: int, th: int = 64, stream=None, **options):
        opt = bfs_options_default()
        opt.th = th
        for k, v in options.items():
            setattr(opt, k, tuple(v) if isinstance(v, list) else v)
        self.opt = opt
        self._h = bfs_build_graph(src, dst, num_vertices, opt, stream)
        self.info = bfs_graph_get_info(self._h)
        self.n = self.info.n

    @property
    def handle(self):
        return self._h

    def set_options(self, **options):
        opt = bfs_options_default()
        for k, v in options.items():
            setattr(opt, k, tuple(v) if isinstance(v, list) else v)
        bfs_set_options(self._h, opt)
        opt.th, opt.edges_on_device = self.opt.th, self.opt.edges_on_device
        self.opt = opt

    def export(self):
        return bfs_graph_export(self._h)

    def run(self, source: int, depth=None, parent=None, stats: bool = False, stream=None):
        """BFS from ``source`` into CUDA tensors (allocated when not given).
        Returns (depth, parent) or (depth, parent, bfs_stats)."""
        import torch

        if depth is None:
            depth = torch.empty(self.n, dtype=torch.int32, device="cuda")
        if parent is None:
            parent = torch.empty(self.n, dtype=torch.int32, device="cuda")
        st = bfs_stats() if stats else None
        bfs_run(self._h, source, depth, parent, st, stream)
        return (depth, parent, st) if stats else (depth, parent)

    def run_many(self, sources, depth=None, parent=None, stream=None):
        """Pipelined runs with results in host memory (pinned tensors allocated when
        not given).  Returns (depth list, parent list, status int32 array)."""
        import torch

        k = len(sources)
        if depth is None:
            depth = [torch.empty(self.n, dtype=torch.int32).pin_memory() for _ in range(k)]
        if parent is None:
            parent = [torch.empty(self.n, dtype=torch.int32).pin_memory() for _ in range(k)]
        status = np.zeros(max(k, 1), dtype=np.int32)
        bfs_run_many(self._h, sources, depth, parent, status, stream)
        return depth, parent, status[:k]

    def wait(self, stream=None):
        bfs_wait(self._h, stream)

    def degree_classes(self, ths, stream=None):
        """Per threshold: delegates and their share of the vertices, and the nn/nd/dn/dd
        shares of the directed entries, in percent (the quantities of Figs. 5 and 7)."""
        st = bfs_degree_class_stats(self._h, ths, stream)
        nnz = max(int(self.info.nnz), 1)
        out = []
        for th, (d, nn, nd, dn, dd) in zip(ths, st.tolist()):
            out.append({"th": int(th), "delegates": d, "delegate_pct": 100.0 * d / self.n,
                        "nn": nn, "nd": nd, "dn": dn, "dd": dd,
                        "nn_pct": 100.0 * nn / nnz, "nd_pct": 100.0 * nd / nnz, "dn_pct": 100.0 * dn / nnz,
                        "dd_pct": 100.0 * dd / nnz})
        return out

    def close(self):
        if getattr(self, "_h", None):
            bfs_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Device state for 64-lane batches of queries on a Graph."""

    def __init__(self, graph: "Graph", with_parents: bool = True, ctas: int = 0):
        self.graph = graph
        self.with_parents = with_parents
        self._h = bfs_batch_create(graph.handle, with_parents, ctas)
        self.device_bytes = bfs_batch_device_bytes(self._h)

    def run(self, sources, depth=None, parent=None, stats: bool = False, stream=None):
        """Runs len(sources) <= 64 queries; returns (depth [k, n] uint8, parent [k, n] int32 or
        None[, stats]) as CUDA tensors (allocated when not given)."""
        import torch

        k = len(sources)
        n = self.graph.n
        if depth is None:
            depth = torch.empty((k, n), dtype=torch.uint8, device="cuda")
        if parent is None and self.with_parents:
            parent = torch.empty((k, n), dtype=torch.int32, device="cuda")
        st = bfs_batch_stats() if stats else None
        bfs_run_batch(self._h, sources, depth, parent, st, stream)
        return (depth, parent, st) if stats else (depth, parent)

    def wait(self, stream=None):
        bfs_batch_wait(self._h, stream)

    def close(self):
        if getattr(self, "_h", None):
            bfs_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching query server over device-resident Graphs (bfs_server_*)."""

    def __init__(self, max_concurrent: int = 2, max_lanes: int = 64, with_parents: bool = True,
                 contexts_per_graph: int = 0, hbm_reserve_bytes: int = 0, hbm_budget_bytes: int = 0,
                 single_path: bool = True, single_max: int = 3, group_batches: bool = True):
        o = bfs_server_options_default()
        o.max_concurrent = max_concurrent
        o.max_lanes = max_lanes
        o.with_parents = 1 if with_parents else 0
        o.contexts_per_graph = contexts_per_graph
        o.hbm_reserve_bytes = hbm_reserve_bytes
        o.hbm_budget_bytes = hbm_budget_bytes
        o.single_path = 1 if single_path else 0
        o.single_max = single_max
        o.group_batches = 1 if group_batches else 0
        self.with_parents = with_parents
        self.graphs = []
        self._live = {}  # ticket -> (depth, parent) kept alive until reported
        self._h = bfs_server_create(o)

    def add_graph(self, graph: "Graph") -> int:
        gid = bfs_server_add_graph(self._h, graph.handle)
        self.graphs.append(graph)
        return gid

    @staticmethod
    def now_ns() -> int:
        return bfs_server_now_ns()

    def submit(self, graph_id: int, source: int, depth=None, parent=None, t_arrival_ns: int = 0) -> int:
        """Queues one query; depth (uint8 [n]) and parent (int32 [n]) are CUDA tensors
        (allocated when not given) that the poll record hands back."""
        import torch

        n = self.graphs[graph_id].n
        if depth is None:
            depth = torch.empty(n, dtype=torch.uint8, device="cuda")
        if parent is None and self.with_parents:
            parent = torch.empty(n, dtype=torch.int32, device="cuda")
        t = bfs_server_submit(self._h, graph_id, source, depth, parent if self.with_parents else None,
                              t_arrival_ns)
        self._live[t] = (depth, parent)
        return t

    def poll(self, timeout_ms: int = 0, max_done: int = 256):
        """Finished queries as dicts (ticket, status, graph_id, batch_size, levels, times,
        depth, parent)."""
        out = []
        for d in bfs_server_poll(self._h, max_done, timeout_ms):
            rec = {f: getattr(d, f) for f, _ in bfs_server_done._fields_}
            rec["depth"], rec["parent"] = self._live.pop(d.ticket, (None, None))
            out.append(rec)
        return out

    def drain(self, timeout_s: float = 120.0):
        """Polls until every submitted query is reported."""
        import time

        out = []
        t_end = time.monotonic() + timeout_s
        while self._live:
            if time.monotonic() > t_end:
                raise TimeoutError("%d queries still outstanding" % len(self._live))
            out += self.poll(timeout_ms=100)
        return out

    def stats(self) -> dict:
        st = bfs_server_get_stats(self._h)
        return {f: getattr(st, f) for f, _ in bfs_server_stats._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            bfs_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats_to_dict(st: bfs_stats) -> dict:
    out = {k: getattr(st, k) for k in ("levels", "logged_levels", "reached", "component_edges",
                                       "edges_examined", "model_bytes", "device_ns", "setup_ns", "result_ns")}
    out["level"] = [{f: getattr(st.level[i], f) for f, _ in bfs_level_log._fields_}
                    for i in range(st.logged_levels)]
    return out
