"""Full-size parity of the batched and serving forms, in the configurations
bench.py times:
  64-lane batches on RMAT scale 24 (edge factor 16, TH 64, the bench's 1024
  seeded sources): one batch with parents, 8 of its lanes compared element by
  element with the oracle (uint8 depth, parent), all 64 lanes with the
  single-source level loop; the bench's autotuned alpha gives the same result;
  the serving mix (RMAT scales 18, 20, 22, 24 and Erdos-Renyi 2^22 with average
  degree 16, one server, Poisson arrivals over the graphs and their sources):
  every query's status is OK, and a sampled 1 % of the queries (at least 3 per
  graph) equal the oracle.
The oracle's host graphs are built in threads while the device works."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import bench
import oracle
from tests.gpu_util import assert_same, need_cuda

pytestmark = pytest.mark.gpu


def _oracle_graph(w):
    hs, hd = bench.make_edges_host(w)
    return oracle.Graph(1 << w["scale"], hs, hd)


def _u8(depth):
    return np.where(depth < 0, 255, depth).astype(np.uint8)


def test_rmat24_batch_full_size():
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    w = bench.WORKLOADS["rmat24"]
    with ThreadPoolExecutor(max_workers=8) as ex:
        fut = ex.submit(_oracle_graph, w)
        g, sources = bench.build_served_graph(w)
        n = g.n
        batch = [int(s) for s in sources[:64]]
        b = bfs.Batch(g, with_parents=True)
        depth = torch.empty((64, n), dtype=torch.uint8, device="cuda")
        parent = torch.empty((64, n), dtype=torch.int32, device="cuda")
        b.run(batch, depth, parent)
        torch.cuda.synchronize()
        b.wait()
        # every lane equals the single-source level loop on the same graph
        d1 = torch.empty(n, dtype=torch.int32, device="cuda")
        p1 = torch.empty(n, dtype=torch.int32, device="cuda")
        for j, s in enumerate(batch):
            g.run(s, d1, p1)
            want_d8 = torch.where(d1 < 0, torch.full_like(d1, 255), d1).to(torch.uint8)
            assert torch.equal(depth[j], want_d8), "lane %d depth differs from the level loop" % j
            assert torch.equal(parent[j], p1), "lane %d parent differs from the level loop" % j
        # 8 lanes against the oracle, one host core each
        og = fut.result()
        lanes = list(range(0, 64, 8))
        want = list(ex.map(lambda j: og.bfs(batch[j]), lanes))
    for j, (wd, wp) in zip(lanes, want):
        assert_same(depth[j].cpu().numpy(), _u8(wd), "lane %d depth (source %d)" % (j, batch[j]))
        assert_same(parent[j].cpu().numpy(), wp, "lane %d parent (source %d)" % (j, batch[j]))
    # the batch schedule the autotuner may pick (alpha) changes no result
    g.set_options(alpha=2)
    d2 = torch.empty((64, n), dtype=torch.uint8, device="cuda")
    p2 = torch.empty((64, n), dtype=torch.int32, device="cuda")
    b.run(batch, d2, p2)
    torch.cuda.synchronize()
    b.wait()
    assert torch.equal(d2, depth) and torch.equal(p2, parent)
    b.close()
    og.close()
    g.close()
    del depth, parent, d2, p2
    torch.cuda.empty_cache()


def test_serving_mix_full_size_sampled():
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    specs = bench.SERVE_GRAPHS
    with ThreadPoolExecutor(max_workers=len(specs) + 8) as ex:
        futs = [ex.submit(_oracle_graph, w) for _, w in specs]
        graphs, sources = [], []
        for _, w in specs:
            g, s = bench.build_served_graph(w)
            graphs.append(g)
            sources.append(s)
        srv = bfs.Server(max_concurrent=2, max_lanes=64, with_parents=True)
        for g in graphs:
            srv.add_graph(g)
        trace = bench.serve_trace(2000, 2000, len(graphs), bench.SERVE_SOURCES, seed=2024)
        rng = np.random.default_rng(7)
        sampled = set(rng.choice(len(trace), size=len(trace) // 100, replace=False).tolist())
        for gid in range(len(graphs)):  # at least three queries of every graph
            sampled.update([i for i, (_, gi, _) in enumerate(trace) if gi == gid][:3])
        t0 = bfs.Server.now_ns() + 2_000_000
        tickets, keep, done, bad = {}, {}, 0, 0

        def collect(recs):  # results of queries not sampled are dropped as they come
            nonlocal done, bad
            for r in recs:
                done += 1
                bad += r["status"] != 0
                i = tickets[r["ticket"]]
                if i in sampled:
                    keep[i] = r

        for i, (off, gid, si) in enumerate(trace):
            while bfs.Server.now_ns() < t0 + off:
                pass
            t = srv.submit(gid, int(sources[gid][si]), t_arrival_ns=t0 + off)
            tickets[t] = i
            collect(srv.poll(timeout_ms=0))
        collect(srv.drain(timeout_s=300))
        assert done == len(trace) and bad == 0, "%d of %d queries reported, %d failed" % (done, len(trace), bad)
        ogs = [f.result() for f in futs]
        jobs = sorted(keep)
        want = list(ex.map(lambda i: ogs[trace[i][1]].bfs(int(sources[trace[i][1]][trace[i][2]])), jobs))
    for i, (wd, wp) in zip(jobs, want):
        _, gid, si = trace[i]
        r = keep[i]
        what = "query %d (graph %s, source %d)" % (i, specs[gid][0], int(sources[gid][si]))
        assert_same(r["depth"].cpu().numpy(), _u8(wd), "depth of " + what)
        assert_same(r["parent"].cpu().numpy(), wp, "parent of " + what)
    srv.close()
    for g in graphs:
        g.close()
    for og in ogs:
        og.close()
    torch.cuda.empty_cache()
