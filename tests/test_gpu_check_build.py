"""The bounds-checked build (-DBFS_CHECK, libbfs_gb300_check.so): every kernel
index it checks (columns, neighbours, queue, chunk-list, long-row and deferred
entries, parent slots, depth words) lies inside its array on one small case per
kernel family, checked on the CPU by the oracle: the direction-optimized level
loop under every schedule and both parent modes, the per-subgraph schedule, the
64-lane batches, the serving loop and the allocation-free entry point.  A
failed check would return BFS_ERR_CHECK (the access is skipped, nothing
traps).  The cases run in a child process that loads the checked library."""
import os
import subprocess
import sys

import pytest

from tests.gpu_util import need_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import graphgen, oracle
import paper_1803_03922_gb300 as bfs
from tests.gpu_util import SCHEDULES, check_against_oracle, gpu_bfs, gpu_graph, assert_same
assert bfs._load()._name.endswith("libbfs_gb300_check.so")
n = 1 << 13
src, dst = graphgen.rmat_host(13, seed=77)
og = oracle.Graph(n, src, dst)
mask = graphgen.nonisolated_mask_host(n, src, dst)
sources = [int(s) for s in graphgen.sample_sources(mask, 6, seed=3)]
e = np.asarray([(i, i + 1) for i in range(300)] + [(0, 400 + k) for k in range(80)], np.int32)
ogp = oracle.Graph(480, e[:, 0], e[:, 1])
for th in (0, 8, 64):
    g = gpu_graph(n, src, dst, th=th)
    gp = gpu_graph(480, e[:, 0], e[:, 1], th=4)
    for name, opts in SCHEDULES.items():
        for tdp in (0, 1):
            g.set_options(td_parent=tdp, **opts)
            check_against_oracle(og, g, sources, stats=True, th=th)
            gp.set_options(td_parent=tdp, **opts)
            check_against_oracle(ogp, gp, [0, 150, 479], stats=True, th=4)
    g.set_options(schedule=6)
    for s in sources:
        d, p = gpu_bfs(g, s)
        wd, wp = og.bfs(s)
        assert_same(d, wd, "subgraph depth"); assert_same(p, wp, "subgraph parent")
    b = bfs.Batch(g)
    bd, bp = b.run(sources)
    wd, wp = og.bfs_batch_u8(sources)
    assert np.array_equal(bd.cpu().numpy(), wd) and np.array_equal(bp.cpu().numpy(), wp)
    b.close()
    g.close()
    gp.close()
g = gpu_graph(n, src, dst, th=16)
srv = bfs.Server(max_concurrent=2)
srv.add_graph(g)
tickets = [srv.submit(0, s) for s in sources * 4]
recs = srv.drain()
assert all(r["status"] == 0 for r in recs)
wd, wp = og.bfs_batch_u8(sources)
for r in recs:
    j = sources.index(sources[(r["ticket"] - 1) % len(sources)])
    assert np.array_equal(r["depth"].cpu().numpy(), wd[j]) and np.array_equal(r["parent"].cpu().numpy(), wp[j])
srv.close()
g.close()
off, col = og.csr()
doff = torch.from_numpy(off).cuda()
dcol = torch.from_numpy(np.concatenate([col, np.zeros(4, np.int32)])).cuda()
for s in sources[:2]:
    d = torch.empty(n, dtype=torch.int32, device="cuda"); p = torch.empty_like(d)
    bfs.bfs_run_static(doff, dcol, n, s, d, p)
    wd, wp = og.bfs(s)
    assert np.array_equal(d.cpu().numpy(), wd) and np.array_equal(p.cpu().numpy(), wp)
print("CHECK-BUILD-OK")
'''


def test_bounds_checked_build_passes():
    need_cuda()
    from paper_1803_03922_gb300 import _build

    lib = _build.build(check=True)
    env = dict(os.environ, BFS_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "CHECK-BUILD-OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
