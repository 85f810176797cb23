"""Serving loop (bfs_server_*): every query's result is the oracle's and is the
same whether the query runs alone or packed with other queries of several graphs;
admission by the memory budget, eviction, lane caps and latency records."""
import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import assert_same, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def _graphs():
    """Small graphs of the serving mix's kinds: RMAT at two scales, uniform random,
    a path (many levels) and several components."""
    out = []
    for scale, th in ((12, 16), (14, 64)):
        src, dst = graphgen.rmat_host(scale, seed=100 + scale)
        out.append((1 << scale, src, dst, th))
    n = 1 << 13
    src, dst = graphgen.er_host(n, n * 8, seed=13)  # average degree 16
    out.append((n, src, dst, 8))
    e = np.array([(i, i + 1) for i in range(199)], np.int32)
    out.append((200, e[:, 0], e[:, 1], 4))
    e = np.array([(0, 1), (1, 2), (10, 11), (11, 12), (12, 13), (20, 21)], np.int32)
    out.append((40, e[:, 0], e[:, 1], 1))
    return out


def _setup(**server_opts):
    need_cuda()
    import paper_1803_03922_gb300 as bfs

    specs = _graphs()
    ogs = [oracle.Graph(n, s, d) for n, s, d, _ in specs]
    gs = [gpu_graph(n, s, d, th=th) for n, s, d, th in specs]
    srv = bfs.Server(**server_opts)
    gids = [srv.add_graph(g) for g in gs]
    assert gids == list(range(len(gs)))
    return bfs, srv, gs, ogs


def _queries(gs, count, seed):
    rng = np.random.default_rng(seed)
    q = []
    for _ in range(count):
        gid = int(rng.integers(0, len(gs)))
        q.append((gid, int(rng.integers(0, gs[gid].n))))
    return q


def _check_oracle(ogs, q, recs, with_parents=True):
    by_graph = {}
    for (gid, s), rec in zip(q, recs):
        by_graph.setdefault(gid, []).append((s, rec))
    for gid, items in by_graph.items():
        for i in range(0, len(items), 64):
            chunk = items[i:i + 64]
            want_d, want_p = ogs[gid].bfs_batch_u8([s for s, _ in chunk])
            for j, (s, rec) in enumerate(chunk):
                assert rec["status"] == 0
                assert_same(rec["depth"].cpu().numpy(), want_d[j], "depth (graph %d, source %d)" % (gid, s))
                if with_parents:
                    assert_same(rec["parent"].cpu().numpy(), want_p[j], "parent (graph %d, source %d)" % (gid, s))


def _run_mix(srv, q):
    tickets = [srv.submit(gid, s) for gid, s in q]
    recs = {r["ticket"]: r for r in srv.drain()}
    return [recs[t] for t in tickets]


def test_mix_equals_alone_and_oracle():
    bfs, srv, gs, ogs = _setup(max_concurrent=2)
    q = _queries(gs, 400, seed=5)
    mix = _run_mix(srv, q)
    _check_oracle(ogs, q, mix)
    st = srv.stats()
    assert st["completed"] == 400 and st["failed"] == 0 and st["waiting"] == 0 and st["in_flight"] == 0
    assert st["launches"] < 400  # queries were packed
    assert max(r["batch_size"] for r in mix) > 1
    # the same queries one at a time through the same server
    for (gid, s), rec in list(zip(q, mix))[::7]:
        t = srv.submit(gid, s)
        (alone,) = srv.drain()
        assert alone["ticket"] == t and alone["batch_size"] == 1
        assert_same(alone["depth"].cpu().numpy(), rec["depth"].cpu().numpy(), "depth alone vs mix")
        assert_same(alone["parent"].cpu().numpy(), rec["parent"].cpu().numpy(), "parent alone vs mix")
    srv.close()


@pytest.mark.parametrize("max_concurrent", [1, 3])
def test_lane_cap_and_concurrency(max_concurrent):
    bfs, srv, gs, ogs = _setup(max_concurrent=max_concurrent, max_lanes=8, contexts_per_graph=1)
    q = _queries(gs, 120, seed=11 + max_concurrent)
    recs = _run_mix(srv, q)
    _check_oracle(ogs, q, recs)
    assert max(r["batch_size"] for r in recs) <= 8
    st = srv.stats()
    assert st["launches"] >= 120 // 8 and st["lanes_launched"] == 120
    assert st["ctas_per_launch"] == st["capacity_ctas"] // max_concurrent
    assert st["contexts_created"] <= len(gs)
    for r in recs:
        assert r["t_arrival_ns"] <= r["t_launch_ns"] <= r["t_done_ns"]
        assert r["device_ns"] > 0 and r["levels"] >= 1
    srv.close()


def test_budget_admission_evicts_idle_contexts():
    need_cuda()
    import paper_1803_03922_gb300 as bfs

    # a budget that holds the largest graph's context but never two of them
    specs = _graphs()
    gs = [gpu_graph(n, s, d, th=th) for n, s, d, th in specs]
    sizes = []
    for g in gs:
        b = bfs.Batch(g)
        sizes.append(b.device_bytes)
        b.close()
    budget = max(sizes) + min(sizes) // 2
    srv = bfs.Server(max_concurrent=1, hbm_budget_bytes=budget, single_path=False)
    ogs = [oracle.Graph(n, s, d) for n, s, d, _ in specs]
    for g in gs:
        srv.add_graph(g)
    q = []
    rng = np.random.default_rng(3)
    for rnd in range(3):  # alternate graphs so contexts keep getting evicted
        for gid in range(len(gs)):
            q += [(gid, int(s)) for s in rng.integers(0, gs[gid].n, 5)]
    recs = []
    for gid, s in q:  # one graph at a time, so each switch needs a new context
        srv.submit(gid, s)
        recs += srv.drain()
    _check_oracle(ogs, q, recs)
    st = srv.stats()
    assert st["contexts_evicted"] > 0
    assert st["context_bytes"] <= budget
    srv.close()


def test_depth_only_server_and_argument_errors():
    bfs, srv, gs, ogs = _setup(with_parents=False, max_concurrent=2)
    q = _queries(gs, 100, seed=21)
    recs = _run_mix(srv, q)
    _check_oracle(ogs, q, recs, with_parents=False)
    import torch

    d = torch.empty(gs[0].n, dtype=torch.uint8, device="cuda")
    p = torch.empty(gs[0].n, dtype=torch.int32, device="cuda")
    for args in ((len(gs), 0, d, None), (0, gs[0].n, d, None), (0, -1, d, None), (0, 0, d, p),
                 (0, 0, np.empty(gs[0].n, np.uint8), None)):
        with pytest.raises(bfs.BfsError) as ex:
            bfs.bfs_server_submit(srv._h, *args)
        assert ex.value.code == bfs.BFS_ERR_INVALID
    srv.close()
    srv2 = bfs.Server()
    with pytest.raises(bfs.BfsError):
        bfs.bfs_server_submit(srv2._h, 0, 0, d, p)  # no graph registered
    srv2.close()


def test_open_loop_arrivals_latency_records():
    """Queries arrive on a schedule (t_arrival in the past or future of the
    submit); latency records are consistent and every result is exact."""
    bfs, srv, gs, ogs = _setup(max_concurrent=2)
    q = _queries(gs, 200, seed=31)
    rng = np.random.default_rng(31)
    t0 = bfs.Server.now_ns()
    gaps = rng.exponential(20_000, len(q)).astype(np.int64)  # 50k queries/s
    arrivals = t0 + np.cumsum(gaps)
    tickets = []
    for (gid, s), ta in zip(q, arrivals):
        while bfs.Server.now_ns() < ta:
            pass
        tickets.append(srv.submit(gid, s, t_arrival_ns=int(ta)))
    recs = {r["ticket"]: r for r in srv.drain()}
    recs = [recs[t] for t in tickets]
    _check_oracle(ogs, q, recs)
    lat = np.array([r["t_done_ns"] - r["t_arrival_ns"] for r in recs])
    assert (lat > 0).all()
    srv.close()


@pytest.mark.parametrize("single_path", [True, False])
def test_lone_queries_and_depth_overflow(single_path):
    """A query that waits alone runs the single-source level loop (uint8 depth,
    same result as the batch form); a depth past 254 is BFS_ERR_OVERFLOW on
    either path, and the server stays usable."""
    bfs, srv, gs, ogs = _setup(max_concurrent=2, single_path=single_path)
    q = _queries(gs, 30, seed=41)
    recs = []
    for gid, s in q:
        srv.submit(gid, s)
        recs += srv.drain()
    _check_oracle(ogs, q, recs)
    st = srv.stats()
    assert st["single_launches"] == (30 if single_path else 0)
    # a few queries of one graph at once: back to back on the level loop while
    # that graph's single-source state is free, else as a batch
    q3 = [(1, int(x)) for x in np.random.default_rng(43).integers(0, gs[1].n, 3)]
    recs3 = _run_mix(srv, q3)
    _check_oracle(ogs, q3, recs3)
    assert (srv.stats()["single_launches"] > 30) == single_path
    e = np.array([(i, i + 1) for i in range(299)], np.int32)  # depth 299 from an end
    deep = gpu_graph(300, e[:, 0], e[:, 1], th=8)
    gid = srv.add_graph(deep)
    srv.submit(gid, 0)
    (r,) = srv.drain()
    assert r["status"] == bfs.BFS_ERR_OVERFLOW
    srv.submit(gid, 150)  # depths <= 150
    (r,) = srv.drain()
    assert r["status"] == 0
    og = oracle.Graph(300, e[:, 0], e[:, 1])
    want_d, want_p = og.bfs_batch_u8([150])
    assert_same(r["depth"].cpu().numpy(), want_d[0], "depth after an overflow")
    assert_same(r["parent"].cpu().numpy(), want_p[0], "parent after an overflow")
    srv.close()


@pytest.mark.parametrize("group", [True, False])
def test_grouped_batches_serve_the_oldest_first(group):
    """With more than max_lanes queries waiting, a grouped batch (the default)
    takes the oldest waiting query and the queries nearest it by the grouping
    key; in arrival order (group_batches off) batches are runs of consecutive
    tickets.  Either way every result equals the oracle."""
    bfs, srv, gs, ogs = _setup(max_concurrent=1, max_lanes=16, group_batches=group)
    rng = np.random.default_rng(21)
    q = [(0, int(s)) for s in rng.integers(0, gs[0].n, 200)]
    tickets = [srv.submit(gid, s) for gid, s in q]
    recs = {r["ticket"]: r for r in srv.drain()}
    _check_oracle(ogs, q, [recs[t] for t in tickets])
    launches = {}
    for t in tickets:
        launches.setdefault(recs[t]["t_launch_ns"], []).append(t)
    remaining = sorted(tickets)
    for t_launch in sorted(launches):
        members = sorted(launches[t_launch])
        assert members[0] == remaining[0], "a launch skipped the oldest waiting query"
        if not group:
            i = remaining.index(members[0])
            assert members == remaining[i:i + len(members)]
        for t in members:
            remaining.remove(t)
        assert len(members) <= 16
    assert not remaining
    srv.close()
