"""The algorithmic byte count behind the roofline: the device's model_bytes of
a run equals the count computed here from the oracle's per-level counters
(frontier size and degree sum, found, scanned, entries examined, queue entries)
for the directions the device took, so the bytes the bench divides by time are
the method's, not a count the kernel could drift from.  bench.py's per-phase
split of the same count must add up to it."""
import numpy as np
import pytest

import bench
import graphgen
import oracle
from tests.gpu_util import gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def _model(og, g, s, st, th):
    info = g.info
    B = 4 * ((info.n_nonisolated + 31) // 32)  # one pass over the visited bitmap
    D = 4 * ((info.delegates + 31) // 32)      # over its delegate prefix
    want_d, _ = og.bfs(s)
    L = st.logged_levels
    dirs = np.array([st.level[i].direction for i in range(L)], dtype=np.int32)
    cnt = og.level_counters(s, want_d, th, dirs)
    b = 8 * info.n  # depth and parent of every vertex
    for i in range(L):
        frontier, mf, found, scanned, edges, _, queue = (int(x) for x in cnt[i])
        if dirs[i] == 0:
            b += 8 * frontier + 8 * mf + 16 * found
        else:
            b += B + 8 * scanned + 8 * edges + 12 * found
        if found > 0:
            b += 2 * (D + B)
            if i + 1 < L and dirs[i + 1] == 0:
                b += 4 * int(cnt[i + 1][6])
    return b


@pytest.mark.parametrize("sched", [dict(schedule=0), dict(schedule=3), dict(schedule=1)],
                         ids=["beamer", "alternate", "topdown"])
def test_model_bytes_from_oracle_counters(sched):
    need_cuda()
    n = 1 << 16
    src, dst = graphgen.rmat_host(16, seed=1616)
    og = oracle.Graph(n, src, dst)
    th = 32
    g = gpu_graph(n, src, dst, th=th, **sched)
    mask = (np.diff(og.csr()[0]) > 0).astype(np.uint8)
    for s in graphgen.sample_sources(mask, 6, seed=16161):
        _, _, st = gpu_bfs(g, int(s), stats=True)
        assert st.model_bytes == _model(og, g, int(s), st, th), "source %d" % s
        info = g.info
        total, phases = bench.algorithmic_bytes(bench.level_list(st), info.n, info.n_nonisolated, info.delegates)
        assert total == st.model_bytes and sum(phases.values()) + 8 * info.n == total
    g.close()
