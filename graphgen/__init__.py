"""Seeded synthetic graph inputs for the BFS path and its oracle.

Input generation only: RMAT (Graph500 quadrant recursion, a,b,c,d = .57,.19,.19,.05,
edge factor 16, ids randomized by a seeded bijection; Sec. VI-A.3 of Pan, Pearce,
Owens, arXiv 1803.03922), Erdos-Renyi pairs, and seeded source sampling.  The
host twin (``gen_host.c``) and the device generator (``gen_device.cu``) share the
arithmetic in ``gg_core.h`` and produce identical edge lists.  Nothing here
computes any part of BFS.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_LIB = os.path.join(_HERE, "libgraphgen_host.so")
_DEV_LIB = os.path.join(_HERE, "libgraphgen_cuda.so")
_host = None
_dev = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)
EDGE_FACTOR = 16


def _stale(out, srcs):
    return not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(s) for s in srcs)


def build_host() -> str:
    srcs = [os.path.join(_HERE, "gen_host.c"), os.path.join(_HERE, "gg_core.h")]
    if _stale(_HOST_LIB, srcs):
        tmp = _HOST_LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-I", _HERE,
                        "-o", tmp, srcs[0]], check=True)
        os.replace(tmp, _HOST_LIB)
    return _HOST_LIB


def build_device_cmd():
    """(output, command) compiling the device generator for sm_103a."""
    src = os.path.join(_HERE, "gen_device.cu")
    tmp = _DEV_LIB + ".tmp%d" % os.getpid()
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC", "-I", _HERE, "-o", tmp, src]
    return tmp, cmd


def build_device() -> str:
    srcs = [os.path.join(_HERE, "gen_device.cu"), os.path.join(_HERE, "gg_core.h")]
    if _stale(_DEV_LIB, srcs):
        tmp, cmd = build_device_cmd()
        subprocess.run(cmd, check=True)
        os.replace(tmp, _DEV_LIB)
    return _DEV_LIB


def _host_lib():
    global _host
    if _host is None:
        lib = ctypes.CDLL(build_host())
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.gg_rmat_host.argtypes = [ctypes.c_int, ctypes.c_int, u64, P, P, ctypes.c_int, ctypes.c_int]
        lib.gg_er_host.argtypes = [i32, i64, u64, P, P, ctypes.c_int]
        lib.gg_perm_host.argtypes = [ctypes.c_int, u64, ctypes.c_uint32]
        lib.gg_perm_host.restype = ctypes.c_uint32
        lib.gg_mark_nonisolated_host.argtypes = [i32, i64, P, P, P]
        lib.gg_mark_nonisolated_host.restype = None
        lib.gg_sample_sources.argtypes = [i32, P, i32, u64, P]
        lib.gg_sample_sources.restype = i32
        _host = lib
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        lib = ctypes.CDLL(build_device())
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.gg_rmat_device.argtypes = [ctypes.c_int, ctypes.c_int, u64, P, P, P]
        lib.gg_er_device.argtypes = [i32, i64, u64, P, P, P]
        lib.gg_mark_nonisolated_device.argtypes = [i64, P, P, P, P]
        _dev = lib
    return _dev


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _threads():
    return max(1, min(64, os.cpu_count() or 1))


def rmat_host(scale: int, seed: int, edge_factor: int = EDGE_FACTOR, permute: bool = True):
    """RMAT edge list on the host: (src, dst) int32 of edge_factor * 2^scale pairs
    (``permute=False`` skips the id bijection, for statistical tests)."""
    m = edge_factor << scale
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _host_lib().gg_rmat_host(scale, edge_factor, seed & (2**64 - 1), _p(src), _p(dst), _threads(),
                                  int(permute))
    if rc:
        raise ValueError("bad RMAT parameters")
    return src, dst


def er_host(n: int, m: int, seed: int):
    """Erdos-Renyi edge list on the host: m uniform pairs on n vertices."""
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _host_lib().gg_er_host(n, m, seed & (2**64 - 1), _p(src), _p(dst), _threads())
    if rc:
        raise ValueError("bad Erdos-Renyi parameters")
    return src, dst


def perm(scale: int, seed: int, x: int) -> int:
    """The seeded id bijection of [0, 2^scale) applied to x."""
    return int(_host_lib().gg_perm_host(scale, seed & (2**64 - 1), x))


def nonisolated_mask_host(n: int, src, dst):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    mask = np.empty(n, dtype=np.uint8)
    _host_lib().gg_mark_nonisolated_host(n, src.size, _p(src), _p(dst), _p(mask))
    return mask


def sample_sources(mask, k: int, seed: int):
    """Seeded uniform sources among vertices with mask[v] != 0, no repeats."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.empty(max(k, 1), dtype=np.int32)
    got = _host_lib().gg_sample_sources(mask.size, _p(mask), k, seed & (2**64 - 1), _p(out))
    return out[:got].copy()


# ---- device generator (torch tensors for memory and streams) --------------------------------

def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def rmat_device(scale: int, seed: int, edge_factor: int = EDGE_FACTOR, device="cuda", stream=None):
    """RMAT edge list generated on the GPU: (src, dst) int32 CUDA tensors."""
    import torch

    m = edge_factor << scale
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    rc = _dev_lib().gg_rmat_device(scale, edge_factor, seed & (2**64 - 1), ctypes.c_void_p(src.data_ptr()),
                                   ctypes.c_void_p(dst.data_ptr()), _stream_ptr(stream))
    if rc:
        raise RuntimeError("gg_rmat_device failed (%d)" % rc)
    return src, dst


def er_device(n: int, m: int, seed: int, device="cuda", stream=None):
    import torch

    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    rc = _dev_lib().gg_er_device(n, m, seed & (2**64 - 1), ctypes.c_void_p(src.data_ptr()),
                                 ctypes.c_void_p(dst.data_ptr()), _stream_ptr(stream))
    if rc:
        raise RuntimeError("gg_er_device failed (%d)" % rc)
    return src, dst


def nonisolated_mask_device(n: int, src, dst, stream=None):
    import torch

    mask = torch.zeros(n, dtype=torch.uint8, device=src.device)
    rc = _dev_lib().gg_mark_nonisolated_device(src.numel(), ctypes.c_void_p(src.data_ptr()),
                                               ctypes.c_void_p(dst.data_ptr()),
                                               ctypes.c_void_p(mask.data_ptr()), _stream_ptr(stream))
    if rc:
        raise RuntimeError("gg_mark_nonisolated_device failed (%d)" % rc)
    return mask
