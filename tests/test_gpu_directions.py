"""Direction decisions of the level loop (Sec. IV-B): for Beamer's alpha/beta rule
and the paper's FV/BV rule, the direction the device takes at every level equals
the oracle's, computed from the exact level sets of the oracle's own BFS.  The
paper rule is evaluated in double on both sides, so the decisions match exactly."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import assert_same, gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu

RULES = [
    ("beamer_stay", dict(alpha=10, beta=18)),
    ("beamer_stay", dict(alpha=15, beta=18)),
    ("beamer_stay", dict(alpha=2, beta=5)),
    ("beamer", dict(alpha=15, beta=18)),
    ("beamer", dict(alpha=2, beta=5)),
    ("beamer", dict(alpha=200, beta=60)),
    ("paper", dict(factor0=0.5, factor1=1e-7)),
    ("paper", dict(factor0=0.05, factor1=0.01)),
    ("paper", dict(factor0=2.0, factor1=0.3)),
]


def _graphs():
    out = []
    src, dst = graphgen.rmat_host(16, seed=116)
    out.append(("rmat16", 1 << 16, src, dst))
    n = 1 << 14
    src, dst = graphgen.er_host(n, n * 4, seed=14)  # average degree 8
    out.append(("er14", n, src, dst))
    e = [(i, i + 1) for i in range(150)] + [(200 + i, 200 + (i + 1) % 40) for i in range(40)]
    e = np.asarray(e, np.int32)
    out.append(("path_and_cycle", 260, e[:, 0], e[:, 1]))
    return out


@pytest.fixture(scope="module")
def graphs():
    need_cuda()
    return [(name, n, src, dst, oracle.Graph(n, src, dst)) for name, n, src, dst in _graphs()]


@pytest.mark.parametrize("rule,params", RULES, ids=["%s-%s" % (r, "-".join("%s" % v for v in p.values()))
                                                    for r, p in RULES])
def test_device_directions_follow_rule(graphs, rule, params):
    for name, n, src, dst, og in graphs:
        opts = dict(schedule={"beamer": 0, "beamer_stay": 7, "paper": 5}[rule], **params)
        g = gpu_graph(n, src, dst, th=16, **opts)
        rng = np.random.default_rng(len(name))
        mask = (np.diff(og.csr()[0]) > 0).astype(np.uint8)
        sources = graphgen.sample_sources(mask, 8, seed=int(rng.integers(1 << 30)))
        for s in sources:
            want_d, _ = og.bfs(int(s))
            d, _, st = gpu_bfs(g, int(s), stats=True)
            assert_same(d, want_d, "depth (%s, source %d)" % (name, s))
            want = og.directions(int(s), want_d, rule, **params)
            assert st.logged_levels == len(want)
            got = [st.level[i].direction for i in range(st.logged_levels)]
            assert got == list(want), "%s %s source %d: device %s oracle %s" % (name, rule, s, got, list(want))
        g.close()
