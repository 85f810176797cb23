"""Pipelined runs with host results (bfs_run_many): every run's depth and parent
equal the oracle's, bit for bit, with page-locked and pageable buffers, an odd
number of runs (both staging slots reused), a buffer pair shared by several
runs (the last run's result lands), isolated sources, and argument errors."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import assert_same, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat():
    need_cuda()
    n = 1 << 14
    src, dst = graphgen.rmat_host(14, seed=141)
    og = oracle.Graph(n, src, dst)
    g = gpu_graph(n, src, dst, th=32)
    mask = (np.diff(og.csr()[0]) > 0).astype(np.uint8)
    sources = [int(s) for s in graphgen.sample_sources(mask, 7, seed=1407)]
    isolated = int(np.flatnonzero(mask == 0)[0]) if (mask == 0).any() else None
    yield n, og, g, sources, isolated
    g.close()


def test_pinned_buffers_match_oracle(rmat):
    n, og, g, sources, isolated = rmat
    srcs = sources + ([isolated] if isolated is not None else [])
    depth, parent, status = g.run_many(srcs)
    assert status.tolist() == [0] * len(srcs)
    for s, d, p in zip(srcs, depth, parent):
        want_d, want_p = og.bfs(s)
        assert_same(d.numpy(), want_d, "depth (source %d)" % s)
        assert_same(p.numpy(), want_p, "parent (source %d)" % s)


def test_pageable_and_shared_buffers(rmat):
    import paper_1803_03922_gb300 as bfs

    n, og, g, sources, _ = rmat
    d = [np.empty(n, np.int32) for _ in sources]
    p = [np.empty(n, np.int32) for _ in sources]
    st = np.zeros(len(sources), np.int32)
    bfs.bfs_run_many(g.handle, sources, d, p, st)
    for s, dd, pp in zip(sources, d, p):
        want_d, want_p = og.bfs(s)
        assert_same(dd, want_d, "depth (pageable, source %d)" % s)
        assert_same(pp, want_p, "parent (pageable, source %d)" % s)
    # one pair for every run: the last run's result is what remains
    import torch

    hd = torch.empty(n, dtype=torch.int32).pin_memory()
    hp = torch.empty(n, dtype=torch.int32).pin_memory()
    k = len(sources)
    bfs.bfs_run_many(g.handle, sources, [hd] * k, [hp] * k)
    want_d, want_p = og.bfs(sources[-1])
    assert_same(hd.numpy(), want_d, "depth (shared buffer)")
    assert_same(hp.numpy(), want_p, "parent (shared buffer)")


def test_same_results_as_single_runs(rmat):
    n, og, g, sources, _ = rmat
    depth, parent, _ = g.run_many(sources[:3])
    for s, d, p in zip(sources[:3], depth, parent):
        d1, p1 = g.run(s)
        assert_same(d.numpy(), d1.cpu().numpy(), "depth vs bfs_run (source %d)" % s)
        assert_same(p.numpy(), p1.cpu().numpy(), "parent vs bfs_run (source %d)" % s)


def test_argument_errors(rmat):
    import torch

    import paper_1803_03922_gb300 as bfs

    n, og, g, sources, _ = rmat
    bfs.bfs_run_many(g.handle, [], [], [])  # no runs: a no-op
    dev = torch.empty(n, dtype=torch.int32, device="cuda")
    host = np.empty(n, np.int32)
    with pytest.raises(bfs.BfsError):
        bfs.bfs_run_many(g.handle, [sources[0]], [dev], [dev])
    with pytest.raises(bfs.BfsError):
        bfs.bfs_run_many(g.handle, [n], [host], [host])
    with pytest.raises(bfs.BfsError):
        bfs.bfs_run_many(g.handle, [-1], [host], [host])
