"""The byte model behind the roofline's achieved bandwidth: the device's
model_bytes of a run equals the model computed here from the oracle's per-level
counters (frontier size and degree sum, found, scanned, entries examined, queue
entries) for the directions the device took, so the bytes the bench divides by
time are the algorithm's, not a count the kernel could drift from."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def _model(og, g, s, st, th):
    info = g.info
    bm = 4 * ((info.n_nonisolated + 31) // 32)  # one pass over a bitmap
    want_d, _ = og.bfs(s)
    L = st.logged_levels
    dirs = np.array([st.level[i].direction for i in range(L)], dtype=np.int32)
    cnt = og.level_counters(s, want_d, th, dirs)
    reached = int((want_d >= 0).sum())
    b = 4 * bm + 12 * info.n + 8 * reached + bm + 4 * info.n_nonisolated  # set-up, results, parent fill
    for i in range(L):
        frontier, mf, found, scanned, edges, _, queue = (int(x) for x in cnt[i])
        fwd = dirs[i] == 0
        if st.level[i].converted:
            b += bm + 4 * queue
        elif fwd and i > 0 and dirs[i - 1] == 1:
            b += 4 * queue  # built by the sparse backward level before
        if fwd:
            b += 20 * frontier + 8 * mf + 12 * found
        else:
            b += bm + 8 * scanned + 8 * edges + 12 * found
        if not (fwd and i == 0) and not (fwd and found == 0):
            b += 4 * bm  # level-end bitmap passes
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
    g.close()
