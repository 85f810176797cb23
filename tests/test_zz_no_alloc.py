"""The allocation-free entry point bfs_run_static, for callers that cannot call
cudaMalloc (code inside another runtime that owns the device allocator, or under
a fixed allocation budget).  Its results must equal the oracle's and bfs_run's,
bit for bit, on consecutive calls that reuse its fixed scratch: RMAT, a long
path, a complete binary tree and a dense random graph with a vertex count that
is not a multiple of 32 (so backward levels and the bitmap tail run), and a
star of the maximum size searched from its centre (one row of 16.7 M entries).
Malformed input is refused with BFS_ERR_INVALID before any row is read, and a
call after a refused one is still correct; sizes beyond its scratch are refused
before anything runs.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle
import paper_1803_03922_gb300 as bfs
from tests.gpu_util import assert_same, gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def _csr(n, src, dst):
    """Symmetric CSR in caller ids, rows ascending, no self-loops or repeats."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keep = src != dst
    s = np.concatenate([src[keep], dst[keep]])
    d = np.concatenate([dst[keep], src[keep]])
    keys = np.unique(s << 32 | d)
    rows = (keys >> 32).astype(np.int64)
    col = (keys & 0xFFFFFFFF).astype(np.int32)
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, rows + 1, 1)
    return np.cumsum(off), col


def _static(torch, doff, dcol, n, s, fill=7):
    lib = bfs._load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    depth = torch.full((n,), fill, dtype=torch.int32, device="cuda")
    parent = torch.full((n,), fill, dtype=torch.int32, device="cuda")
    rc = lib.bfs_run_static(ctypes.c_void_p(doff.data_ptr()), ctypes.c_void_p(dcol.data_ptr()), n, int(s),
                            ctypes.c_void_p(depth.data_ptr()), ctypes.c_void_p(parent.data_ptr()), stream)
    return rc, depth, parent


def _graphs():
    out = []
    # RMAT scale 14 (n a multiple of 32)
    n = 1 << 14
    src, dst = graphgen.rmat_host(14, seed=41)
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    out.append(("rmat14", n, src, dst, [int(x) for x in graphgen.sample_sources(mask, 2, seed=5)]))
    # a path of 1000 vertices (ragged n, 999 levels), from an end and from the middle
    n = 1000
    out.append(("path1000", n, np.arange(n - 1), np.arange(1, n), [0, 517]))
    # a complete binary tree in heap order (ragged n), from the root and a leaf
    n = 2000
    v = np.arange(1, n)
    out.append(("tree2000", n, (v - 1) // 2, v, [0, n - 1]))
    # a dense random graph with ragged n: backward levels do most of the work
    n = 3001
    rng = np.random.default_rng(3)
    m = n * 20
    out.append(("er3001", n, rng.integers(0, n, m), rng.integers(0, n, m), [0, 1234]))
    return out


def test_static_entry_point_matches_oracle_and_bfs_run():
    torch = need_cuda()
    saw_backward = False
    for name, n, src, dst, sources in _graphs():
        off, col = _csr(n, src, dst)
        doff = torch.from_numpy(off).cuda()
        dcol = torch.from_numpy(np.concatenate([col, np.zeros(4, np.int32)])).cuda()
        og = oracle.Graph(n, np.asarray(src, np.int32), np.asarray(dst, np.int32))
        g = gpu_graph(n, np.asarray(src, np.int32), np.asarray(dst, np.int32), th=16)
        for s in sources:  # calls in a row share the fixed scratch
            rc, depth, parent = _static(torch, doff, dcol, n, s)
            assert rc == bfs.BFS_OK, bfs.bfs_last_error()
            want_d, want_p = og.bfs(int(s))
            assert_same(depth.cpu().numpy(), want_d, "%s depth (source %d)" % (name, s))
            assert_same(parent.cpu().numpy(), want_p, "%s parent (source %d)" % (name, s))
            d2, p2 = gpu_bfs(g, int(s))
            assert_same(d2, want_d, "%s bfs_run depth" % name)
            assert_same(p2, want_p, "%s bfs_run parent" % name)
            # the same Beamer rule (alpha 15, beta 18) takes these directions
            saw_backward |= bool(og.directions(int(s), want_d, "beamer").any())
        g.close()
        og.close()
    assert saw_backward, "no graph of this test takes a backward level"


def test_static_entry_point_isolated_source_through_binding():
    torch = need_cuda()
    n = 1 << 12
    src, dst = graphgen.rmat_host(12, seed=9)
    off, col = _csr(n, src, dst)
    doff = torch.from_numpy(off).cuda()
    dcol = torch.from_numpy(np.concatenate([col, np.zeros(4, np.int32)])).cuda()
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    iso = int(np.flatnonzero(mask == 0)[0])
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_run_static(doff, dcol, n, iso, depth, parent)
    want_d = np.full(n, -1, np.int32)
    want_d[iso] = 0
    want_p = np.full(n, -1, np.int32)
    want_p[iso] = iso
    assert_same(depth.cpu().numpy(), want_d, "isolated source depth")
    assert_same(parent.cpu().numpy(), want_p, "isolated source parent")


def test_static_entry_point_largest_star_from_centre():
    """Star of 2^24 vertices from its centre: the centre's row (16,777,215
    entries) is walked in one forward level; depth 1 and parent = centre for
    every leaf (closed form), well inside the barrier bound."""
    torch = need_cuda()
    n = 1 << 24
    c = 12345
    leaves = np.concatenate([np.arange(c), np.arange(c + 1, n)]).astype(np.int32)
    off = np.empty(n + 1, np.int64)
    off[0] = 0
    deg = np.ones(n, np.int64)
    deg[c] = n - 1
    off[1:] = np.cumsum(deg)
    col = np.empty(2 * (n - 1), np.int32)
    # rows in ascending vertex order: leaves before the centre, the centre, leaves after
    col[:c] = c
    col[c:c + n - 1] = leaves
    col[c + n - 1:] = c
    doff = torch.from_numpy(off).cuda()
    dcol = torch.from_numpy(col).cuda()
    for s in (c, 0):
        rc, depth, parent = _static(torch, doff, dcol, n, s)
        assert rc == bfs.BFS_OK, bfs.bfs_last_error()
        d = depth.cpu().numpy()
        p = parent.cpu().numpy()
        if s == c:
            want_d = np.ones(n, np.int32)
            want_d[c] = 0
            want_p = np.full(n, c, np.int32)
        else:  # from a leaf: the centre at depth 1, the other leaves at depth 2 through it
            want_d = np.full(n, 2, np.int32)
            want_d[c] = 1
            want_d[0] = 0
            want_p = np.full(n, c, np.int32)
            want_p[c] = 0
            want_p[0] = 0
        assert_same(d, want_d, "star depth from %d" % s)
        assert_same(p, want_p, "star parent from %d" % s)
    del doff, dcol
    torch.cuda.empty_cache()


def test_static_entry_point_refuses_malformed_csr_then_recovers():
    torch = need_cuda()
    n = 1000
    off, col = _csr(n, np.arange(n - 1), np.arange(1, n))
    og = oracle.Graph(n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32))
    want_d, want_p = og.bfs(3)
    bad_col = col.copy()
    bad_col[777] = n + 5
    bad_off = off.copy()
    bad_off[400] = bad_off[402] + 1
    neg_col = col.copy()
    neg_col[10] = -1
    for o, c, what in ((off, bad_col, "column past n"), (bad_off, col, "offsets decreasing"),
                       (off, neg_col, "negative column")):
        doff = torch.from_numpy(o).cuda()
        dcol = torch.from_numpy(c).cuda()
        rc, _, _ = _static(torch, doff, dcol, n, 3)
        assert rc == bfs.BFS_ERR_INVALID, "%s: rc %d" % (what, rc)
        # the next call with a good graph is correct (the scratch carries nothing over)
        rc, depth, parent = _static(torch, torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda(), n, 3)
        assert rc == bfs.BFS_OK, bfs.bfs_last_error()
        assert_same(depth.cpu().numpy(), want_d, "depth after a refused call")
        assert_same(parent.cpu().numpy(), want_p, "parent after a refused call")
    og.close()


def test_static_entry_point_refuses_host_pointers_and_oversize():
    torch = need_cuda()
    lib = bfs._load()
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.bfs_run_static(p, p, (1 << 24) + 1, 0, p, p, None)
    assert rc == bfs.BFS_ERR_OVERFLOW
    assert "16777216" in bfs.bfs_last_error()
    host = np.zeros(16, np.int64)
    hp = ctypes.c_void_p(host.ctypes.data)
    rc = lib.bfs_run_static(hp, p, 4, 0, p, p, None)
    assert rc == bfs.BFS_ERR_INVALID
    rc = lib.bfs_run_static(p, p, 4, 0, hp, p, None)
    assert rc == bfs.BFS_ERR_INVALID
