"""Per-subgraph directions (Sec. IV-B; BFS_SCHED_PAPER_SUBGRAPH): the dd, dn and
nd visits each switch by the FV/BV rule with their own factor pair while nn
stays forward.  At every level the three directions the device takes equal the
oracle's (orc_subgraph_directions, computed from the exact level sets of the
oracle's own BFS, in double on both sides), and depth and parent equal the
oracle's bit for bit: a direction changes the work, never the output."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.golden_io import read_subgraph_directions
from tests.gpu_util import assert_same, gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu

FACTORS = [
    ((0.5, 0.05, 1e-7), (1e-7, 1e-7, 1e-7)),  # the paper's values (Sec. VI-B)
    ((2.0, 0.5, 0.01), (0.3, 0.3, 0.3)),      # later switches, and switching back
    ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),       # every subgraph backward at its first frontier
    ((0.05, 5.0, 0.5), (10.0, 0.01, 2.0)),
]


def _graphs():
    out = []
    src, dst = graphgen.rmat_host(16, seed=116)
    out.append(("rmat16", 1 << 16, src, dst, 16))
    src, dst = graphgen.rmat_host(14, seed=77)
    out.append(("rmat14_th4", 1 << 14, src, dst, 4))
    n = 1 << 13
    src, dst = graphgen.er_host(n, n * 6, seed=13)  # average degree 12, th 12: both classes
    out.append(("er13", n, src, dst, 12))
    e = [(i, i + 1) for i in range(150)] + [(200 + i, 200 + (i + 1) % 40) for i in range(40)] + \
        [(300, 300 + k) for k in range(1, 60)]
    e = np.asarray(e, np.int32)
    out.append(("path_cycle_star", 371, e[:, 0], e[:, 1], 2))
    return out


@pytest.fixture(scope="module")
def graphs():
    need_cuda()
    return [(name, n, src, dst, th, oracle.Graph(n, src, dst)) for name, n, src, dst, th in _graphs()]


def _check(g, og, s, th, f0, f1, what):
    want_d, want_p = og.bfs(int(s))
    d, p, st = gpu_bfs(g, int(s), stats=True)
    assert_same(d, want_d, "depth (%s, source %d)" % (what, s))
    assert_same(p, want_p, "parent (%s, source %d)" % (what, s))
    want = og.subgraph_directions(int(s), want_d, th, f0, f1)
    assert st.logged_levels == len(want), "%s: %d levels, oracle %d" % (what, st.logged_levels, len(want))
    got = [st.level[i].subgraph_directions for i in range(st.logged_levels)]
    assert got == list(want), "%s source %d: device %s oracle %s" % (what, s, got, list(want))
    assert [st.level[i].direction for i in range(st.logged_levels)] == [int(x != 0) for x in want]
    return got


@pytest.mark.parametrize("f0,f1", FACTORS, ids=["f%d" % i for i in range(len(FACTORS))])
def test_device_subgraph_directions_follow_rule(graphs, f0, f1):
    seen = set()
    for name, n, src, dst, th, og in graphs:
        g = gpu_graph(n, src, dst, th=th, schedule=6)
        g.set_options(schedule=6, subgraph_factor0=f0, subgraph_factor1=f1)
        mask = (og.degree() > 0).astype(np.uint8)
        sources = graphgen.sample_sources(mask, 6, seed=len(name) * 31 + 7)
        for s in sources:
            seen.update(_check(g, og, s, th, f0, f1, name))
        g.close()
    assert len(seen) > 1, "the factors gave one direction pattern only: %s" % sorted(seen)


def test_hand_worked_graphs_on_device():
    """The graphs of tests/golden/subgraph_directions_worked.txt run on the device."""
    need_cuda()
    graphs, cases = read_subgraph_directions()
    for gname, src, f0, f1, want in cases:
        n, th, s, d = graphs[gname]
        og = oracle.Graph(n, s, d)
        g = gpu_graph(n, s, d, th=th)
        g.set_options(schedule=6, subgraph_factor0=f0, subgraph_factor1=f1)
        got = _check(g, og, src, th, f0, f1, gname)
        assert got == want
        g.close()


def test_rmat22_subgraph_schedule_full_size():
    """RMAT scale 22 at TH 64 (the benchmark's graph of that scale), the paper's
    factors: two sources against the oracle, directions included."""
    torch = need_cuda()
    import bench

    w = bench.WORKLOADS["rmat22"]
    n = 1 << w["scale"]
    hs, hd = bench.make_edges_host(w)
    og = oracle.Graph(n, hs, hd)
    mask = graphgen.nonisolated_mask_host(n, hs, hd)
    sources = bench.sources_for(w, mask)
    g = gpu_graph(n, hs, hd, th=w["th"])
    del hs, hd
    g.set_options(schedule=6)
    for s in sources[:2]:
        _check(g, og, s, w["th"], (0.5, 0.05, 1e-7), (1e-7, 1e-7, 1e-7), "rmat22")
    g.close()
    og.close()
    torch.cuda.empty_cache()
