"""Parity at the benchmark's full size, in the configuration bench.py times:
RMAT scale 22 (edge factor 16, a,b,c,d = .57,.19,.19,.05, ids permuted), TH 64,
the same 64 seeded sources, device-generated edges, default options.  16 of the
sources are compared element by element with the oracle (depth, parent, the
component edge count and every per-level counter); all 64 must give identical
results for every TH of the sweep and for forced schedules (Sec. IV-B: the
direction never changes the output).  Scale 26 (the largest benchmark graph) is
compared on two sources when BFS_RUN_SLOW=1."""
import os

import numpy as np
import pytest

import bench
import graphgen
import oracle
from tests.gpu_util import assert_same, check_counters, need_cuda

pytestmark = pytest.mark.gpu


def _setup(name):
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    w = bench.WORKLOADS[name]
    n = 1 << w["scale"]
    src, dst = graphgen.rmat_device(w["scale"], seed=w["seed"])
    mask = graphgen.nonisolated_mask_device(n, src, dst).cpu().numpy()
    sources = bench.sources_for(w, mask)
    hs, hd = graphgen.rmat_host(w["scale"], seed=w["seed"])
    og = oracle.Graph(n, hs, hd)
    del hs, hd
    g = bfs.Graph(src, dst, n, th=w["th"])
    return torch, bfs, w, n, src, dst, sources, og, g


@pytest.fixture(scope="module")
def rmat22():
    return _setup("rmat22")


def _run(g, torch, s, stats=False):
    out = g.run(int(s), stats=stats)
    torch.cuda.synchronize()
    return (out[0].cpu().numpy(), out[1].cpu().numpy()) + ((out[2],) if stats else ())


def test_rmat22_sampled_sources_bit_exact(rmat22):
    torch, bfs, w, n, src, dst, sources, og, g = rmat22
    for s in sources[::4]:
        d, p, st = _run(g, torch, s, stats=True)
        want_d, want_p = og.bfs(int(s))
        assert_same(d, want_d, "depth (source %d)" % s)
        assert_same(p, want_p, "parent (source %d)" % s)
        assert st.component_edges == og.component_edges(want_d)
        assert st.reached == int((want_d >= 0).sum())
        check_counters(og, s, want_d, st, w["th"], pull=g.opt.td_parent == 0)


def test_rmat22_all_sources_th_and_schedule_invariant(rmat22):
    torch, bfs, w, n, src, dst, sources, og, g = rmat22
    ref = {int(s): _run(g, torch, s) for s in sources}
    for th in (32, 128, 256):
        g2 = bfs.Graph(src, dst, n, th=th)
        for s in sources:
            d, p = _run(g2, torch, s)
            assert_same(d, ref[int(s)][0], "depth th=%d source %d" % (th, s))
            assert_same(p, ref[int(s)][1], "parent th=%d source %d" % (th, s))
        g2.close()
    for sched in (1, 2, 5):
        g.set_options(schedule=sched)
        for s in sources[::8]:
            d, p = _run(g, torch, s)
            assert_same(d, ref[int(s)][0], "depth schedule=%d" % sched)
            assert_same(p, ref[int(s)][1], "parent schedule=%d" % sched)
    g.set_options()


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("BFS_RUN_SLOW") != "1", reason="scale-26 oracle comparison: set BFS_RUN_SLOW=1")
def test_rmat26_two_sources_bit_exact():
    torch, bfs, w, n, src, dst, sources, og, g = _setup("rmat26")
    for s in sources[:2]:
        d, p, st = _run(g, torch, s, stats=True)
        want_d, want_p = og.bfs(int(s))
        assert_same(d, want_d, "depth (source %d)" % s)
        assert_same(p, want_p, "parent (source %d)" % s)
        assert st.component_edges == og.component_edges(want_d)
