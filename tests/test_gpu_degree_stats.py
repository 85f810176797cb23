"""Degree-class statistics (Sec. VI-B, Figs. 5 and 7) from the device histograms
equal the oracle's separation and subgraph counts for every threshold, and the
same graph's separation at its own TH agrees with its build-time counts."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import gpu_graph, need_cuda

pytestmark = pytest.mark.gpu

THS = [0, 1, 2, 3, 5, 8, 16, 31, 64, 100, 1023, 1024, 1025, 4096, 10 ** 9]


def _cases():
    src, dst = graphgen.rmat_host(15, seed=115)
    yield "rmat15", 1 << 15, src, dst
    n = 1 << 12
    src, dst = graphgen.er_host(n, n * 6, seed=12)
    yield "er12", n, src, dst
    # a hub of degree 3000 (above the shared-memory bins), leaves, isolated vertices
    e = np.asarray([(0, x) for x in range(1, 3001)] + [(1, 2), (5, 6)], np.int32)
    yield "hub", 3100, e[:, 0], e[:, 1]


@pytest.mark.parametrize("name,n,src,dst", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_degree_class_stats_match_oracle(name, n, src, dst):
    need_cuda()
    import paper_1803_03922_gb300 as bfs

    og = oracle.Graph(n, src, dst)
    g = gpu_graph(n, src, dst, th=64)
    got = bfs.bfs_degree_class_stats(g.handle, THS)
    for i, th in enumerate(THS):
        _, _, d, _ = og.separate(th)
        want = [d] + [int(x) for x in og.subgraph_counts(th)]
        assert got[i].tolist() == want, "%s th=%d: device %s oracle %s" % (name, th, got[i].tolist(), want)
    # at the graph's own threshold the sweep agrees with the build's counts
    i64 = THS.index(64)
    assert got[i64][0] == g.info.delegates
    assert got[i64][1:].tolist() == list(g.info.subgraph_edges)
    rows = g.degree_classes(THS)
    assert abs(sum(rows[3][k] for k in ("nn_pct", "nd_pct", "dn_pct", "dd_pct")) - 100.0) < 1e-9
    with pytest.raises(bfs.BfsError):
        bfs.bfs_degree_class_stats(g.handle, [-1])
    g.close()
