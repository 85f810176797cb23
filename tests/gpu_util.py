"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle

SCHEDULES = {
    "beamer": dict(schedule=0),
    "beamer_stay": dict(schedule=7),
    "topdown": dict(schedule=1),
    "bottomup": dict(schedule=2),
    "alternate": dict(schedule=3),
    "paper": dict(schedule=5),
}


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_graph(n, src, dst, th=64, device_edges=False, **opts):
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    if device_edges:
        s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda()
        d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda()
    else:
        s = np.ascontiguousarray(src, np.int32)
        d = np.ascontiguousarray(dst, np.int32)
    return bfs.Graph(s, d, n, th=th, **opts)


def gpu_bfs(g, source, stats=False):
    out = g.run(source, stats=stats)
    d = out[0].cpu().numpy()
    p = out[1].cpu().numpy()
    return (d, p, out[2]) if stats else (d, p)


def assert_same(a, b, what):
    if not np.array_equal(a, b):
        bad = np.flatnonzero(a != b)
        raise AssertionError("%s differs at %d positions, first %s: got %s want %s" %
                             (what, bad.size, bad[:5].tolist(), a[bad[:5]].tolist(), b[bad[:5]].tolist()))


def check_against_oracle(og: oracle.Graph, g, sources, stats=False, th=None):
    for s in sources:
        want_d, want_p = og.bfs(int(s))
        res = gpu_bfs(g, int(s), stats=stats)
        assert_same(res[0], want_d, "depth (source %d)" % s)
        assert_same(res[1], want_p, "parent (source %d)" % s)
        if stats:
            st = res[2]
            assert st.levels == int(want_d.max()) + 1
            assert st.component_edges == og.component_edges(want_d)
            assert st.reached == int((want_d >= 0).sum())
            if th is not None:
                check_counters(og, s, want_d, st, th, pull=g.opt.td_parent == 0)


def check_counters(og, s, depth, st, th, pull=True):
    """Per-level device counters equal the oracle's, for the directions the device took."""
    L = st.logged_levels
    dirs = np.array([st.level[i].direction for i in range(L)], dtype=np.int32)
    want = og.level_counters(int(s), depth, th, dirs)
    for i in range(L):
        lv = st.level[i]
        got = [lv.frontier, lv.frontier_edges, lv.found,
               lv.scanned if dirs[i] == 1 else 0, lv.edges_examined if dirs[i] == 1 else 0,
               lv.parent_edges if (dirs[i] == 0 and pull) else 0, lv.queue_entries if dirs[i] == 0 else 0]
        w = list(want[i])
        if not pull:
            w[5] = 0
        if dirs[i] == 1:
            w[6] = 0
        assert got == w, "level %d counters %s, oracle %s" % (i, got, w)
