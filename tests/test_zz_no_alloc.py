"""The allocation-free entry point bfs_run_static, for callers that cannot call
cudaMalloc (code inside another runtime that owns the device allocator, or under
a fixed allocation budget).  It must give the same depth and parent as bfs_run,
bit for bit, on consecutive calls that reuse its fixed scratch; sizes beyond its
scratch are refused before anything runs.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_1803_03922_gb300 as bfs
from tests.gpu_util import gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def _csr(n, src, dst):
    """Symmetric CSR in caller ids, rows ascending, no self-loops or repeats."""
    keep = src != dst
    s = np.concatenate([src[keep], dst[keep]]).astype(np.int64)
    d = np.concatenate([dst[keep], src[keep]]).astype(np.int64)
    keys = np.unique(s << 32 | d)
    rows = (keys >> 32).astype(np.int64)
    col = (keys & 0xFFFFFFFF).astype(np.int32)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, rows + 1, 1)
    return np.cumsum(off), col


def test_static_entry_point_matches_bfs_run():
    torch = need_cuda()
    scale = 14
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=41)
    off, col = _csr(n, src, dst)
    doff = torch.from_numpy(off).cuda()
    dcol = torch.from_numpy(np.concatenate([col, np.zeros(4, np.int32)])).cuda()
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    sources = graphgen.sample_sources(mask, 2, seed=5)
    g = gpu_graph(n, src, dst, th=64)
    lib = bfs._load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for s in sources:  # two calls in a row share the fixed scratch
        depth = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        parent = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        rc = lib.bfs_run_static(ctypes.c_void_p(doff.data_ptr()), ctypes.c_void_p(dcol.data_ptr()), n, int(s),
                                ctypes.c_void_p(depth.data_ptr()), ctypes.c_void_p(parent.data_ptr()), stream)
        assert rc == bfs.BFS_OK, bfs.bfs_last_error()
        want_d, want_p = gpu_bfs(g, int(s))
        assert np.array_equal(depth.cpu().numpy(), want_d)
        assert np.array_equal(parent.cpu().numpy(), want_p)
    # an isolated source through the binding of the same name
    iso = int(np.flatnonzero(mask == 0)[0])
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_run_static(doff, dcol, n, iso, depth, parent)
    want_d, want_p = gpu_bfs(g, iso)
    assert np.array_equal(depth.cpu().numpy(), want_d) and np.array_equal(parent.cpu().numpy(), want_p)


def test_static_entry_point_refuses_oversize():
    torch = need_cuda()
    lib = bfs._load()
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.bfs_run_static(p, p, (1 << 24) + 1, 0, p, p, None)
    assert rc == bfs.BFS_ERR_OVERFLOW
    assert "16777216" in bfs.bfs_last_error()
