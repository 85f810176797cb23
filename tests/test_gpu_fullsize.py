"""Parity at the benchmark's full sizes, in the configuration bench.py times:
device-generated edges, default options, the same 64 seeded sources.

  RMAT scale 26 (the benchmark workload; edge factor 16, a,b,c,d =
  .57,.19,.19,.05, ids permuted), TH 64: four sources compared element by
  element with the oracle (depth, parent, component edge count, reached count and
  every per-level counter); all 64 sources identical for TH 16 (the per-scale
  rule), 64 and 256 and for forced schedules (Sec. IV-B: a direction changes the
  work, never the output).
  Erdos-Renyi 2^26 vertices, average degree 32: four sources against the oracle.
  RMAT scale 22, TH 64: 16 sources against the oracle, all 64 over the TH sweep.

The oracle runs on the host, one single-threaded run per source, several at a
time on separate cores."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import bench
import graphgen
import oracle
from tests.gpu_util import assert_same, check_counters, need_cuda

pytestmark = pytest.mark.gpu


def _oracle_graph(name):
    w = bench.WORKLOADS[name]
    hs, hd = bench.make_edges_host(w)
    return oracle.Graph(1 << w["scale"], hs, hd)


# The oracle's host graphs of the two scale-26 workloads take minutes each to
# build on one core: both start together, in threads, on first use.
_POOL = ThreadPoolExecutor(max_workers=2)
_ORACLES = {}


def _oracle_future(name):
    if name not in _ORACLES:
        _ORACLES[name] = _POOL.submit(_oracle_graph, name)
    return _ORACLES[name]


def _setup(name, th=None):
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    if name in ("rmat26", "er26"):
        _oracle_future("rmat26")
        _oracle_future("er26")
    fut = _oracle_future(name)
    w = bench.WORKLOADS[name]
    n = 1 << w["scale"]
    src, dst = bench.make_edges_device(w)
    mask = graphgen.nonisolated_mask_device(n, src, dst).cpu().numpy()
    sources = bench.sources_for(w, mask)
    g = bfs.Graph(src, dst, n, th=w["th"] if th is None else th)
    torch.cuda.synchronize()
    og = fut.result()
    _ORACLES.pop(name, None)
    return torch, bfs, w, n, src, dst, sources, og, g


def _run(g, torch, s, stats=False):
    out = g.run(int(s), stats=stats)
    torch.cuda.synchronize()
    return (out[0].cpu().numpy(), out[1].cpu().numpy()) + ((out[2],) if stats else ())


def _oracle_many(og, sources):
    with ThreadPoolExecutor(max_workers=len(sources)) as ex:
        return list(ex.map(lambda s: og.bfs(int(s)), sources))


def _compare_with_oracle(torch, g, og, w, sources):
    want = _oracle_many(og, sources)
    for s, (want_d, want_p) in zip(sources, want):
        d, p, st = _run(g, torch, s, stats=True)
        assert_same(d, want_d, "depth (source %d)" % s)
        assert_same(p, want_p, "parent (source %d)" % s)
        assert st.component_edges == og.component_edges(want_d)
        assert st.reached == int((want_d >= 0).sum())
        assert st.levels == int(want_d.max()) + 1
        check_counters(og, s, want_d, st, w["th"], pull=g.opt.td_parent == 0)


def _same_on_device(torch, g_ref, g, s, what):
    d0, p0 = g_ref.run(int(s))
    d1, p1 = g.run(int(s))
    if not (torch.equal(d0, d1) and torch.equal(p0, p1)):
        a, b = _run(g, torch, s)
        assert_same(a, d0.cpu().numpy(), "depth %s source %d" % (what, s))
        assert_same(b, p0.cpu().numpy(), "parent %s source %d" % (what, s))


@pytest.fixture(scope="module")
def rmat26():
    ctx = _setup("rmat26")
    yield ctx
    ctx[8].close()
    ctx[7].close()


@pytest.fixture(scope="module")
def rmat22():
    ctx = _setup("rmat22")
    yield ctx
    ctx[8].close()
    ctx[7].close()


def test_rmat26_four_sources_bit_exact(rmat26):
    torch, bfs, w, n, src, dst, sources, og, g = rmat26
    _compare_with_oracle(torch, g, og, w, sources[:4])


def test_rmat26_all_sources_th_and_schedule_invariant(rmat26):
    torch, bfs, w, n, src, dst, sources, og, g = rmat26
    for th in (16, 256):
        g2 = bfs.Graph(src, dst, n, th=th)
        for s in sources:
            _same_on_device(torch, g, g2, s, "th=%d" % th)
        g2.close()
        torch.cuda.empty_cache()
    for sched in (1, 2, 5):
        g2 = bfs.Graph(src, dst, n, th=w["th"], schedule=sched)
        for s in sources[::8]:
            _same_on_device(torch, g, g2, s, "schedule=%d" % sched)
        g2.close()
        torch.cuda.empty_cache()


def test_er26_four_sources_bit_exact():
    torch, bfs, w, n, src, dst, sources, og, g = _setup("er26")
    try:
        _compare_with_oracle(torch, g, og, w, sources[:4])
    finally:
        g.close()
        og.close()


def test_rmat22_sampled_sources_bit_exact(rmat22):
    torch, bfs, w, n, src, dst, sources, og, g = rmat22
    _compare_with_oracle(torch, g, og, w, sources[::4])


def test_rmat22_all_sources_th_and_schedule_invariant(rmat22):
    torch, bfs, w, n, src, dst, sources, og, g = rmat22
    for th in (32, 128, 256):
        g2 = bfs.Graph(src, dst, n, th=th)
        for s in sources:
            _same_on_device(torch, g, g2, s, "th=%d" % th)
        g2.close()
    for sched in (1, 2, 5):
        g2 = bfs.Graph(src, dst, n, th=w["th"], schedule=sched)
        for s in sources[::8]:
            _same_on_device(torch, g, g2, s, "schedule=%d" % sched)
        g2.close()
