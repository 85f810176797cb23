"""CUDA path vs the CPU oracle, element by element (bit-exact depth and parent),
through the C ABI.  Inputs are seeded: closed-form graphs, random graphs with
ragged vertex counts, and RMAT graphs (a,b,c,d = .57,.19,.19,.05, edge factor 16,
ids permuted; Sec. VI-A.3)."""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import SCHEDULES, check_against_oracle, gpu_bfs, gpu_graph, need_cuda, assert_same

pytestmark = pytest.mark.gpu


def _closed_form_graphs():
    g = {}
    n = 37
    g["path"] = (n, [(i, i + 1) for i in range(n - 1)], [0, 18, 36])
    g["star"] = (70, [(13, v) for v in range(70) if v != 13], [13, 40])
    R, C = 9, 13
    e = []
    for r in range(R):
        for c in range(C):
            if r + 1 < R:
                e.append((r * C + c, (r + 1) * C + c))
            if c + 1 < C:
                e.append((r * C + c + 1, r * C + c))
    g["grid"] = (R * C, e, [0, 60])
    g["bintree"] = (255, [((i - 1) // 2, i) for i in range(1, 255)], [0, 100])
    g["complete"] = (40, list(itertools.combinations(range(40), 2)), [5])
    g["cycle"] = (66, [(i, (i + 1) % 66) for i in range(66)], [0, 33])
    g["components"] = (75, [(0, 1), (1, 2), (40, 41), (41, 42), (42, 43), (70, 71)], [41, 74, 0])
    g["single"] = (1, [], [0])
    g["no_edges"] = (33, [], [32])
    g["loops_dups"] = (5, [(0, 0), (0, 1), (1, 0), (0, 1), (1, 2), (2, 2), (4, 4)], [0, 4])
    return g


@pytest.mark.parametrize("name", list(_closed_form_graphs().keys()))
@pytest.mark.parametrize("th", [0, 2, 64, 10**9])
def test_closed_forms_all_schedules(name, th):
    n, e, sources = _closed_form_graphs()[name]
    e = np.asarray(e, dtype=np.int32).reshape(-1, 2)
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th)
    for sched, opts in SCHEDULES.items():
        for tdp in (0, 1):
            g.set_options(td_parent=tdp, **opts)
            check_against_oracle(og, g, sources, stats=True, th=th)


def test_random_small_graphs():
    rng = np.random.default_rng(2024)
    for trial in range(60):
        n = int(rng.integers(1, 400))
        m = int(rng.integers(0, 6 * n))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        if m and trial % 3 == 0:
            src[: m // 4] = int(rng.integers(0, n))  # a hub
        og = oracle.Graph(n, src, dst)
        th = int(rng.choice([0, 1, 3, 8, 64]))
        g = gpu_graph(n, src, dst, th=th, device_edges=bool(trial & 1))
        sched = list(SCHEDULES.values())[trial % len(SCHEDULES)]
        g.set_options(td_parent=trial % 2, **sched)
        sources = rng.integers(0, n, 3)
        check_against_oracle(og, g, sources, stats=True, th=th)


def test_random_schedule_masks():
    src, dst = graphgen.rmat_host(12, seed=77)
    n = 1 << 12
    og = oracle.Graph(n, src, dst)
    g = gpu_graph(n, src, dst, th=16)
    rng = np.random.default_rng(5)
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    sources = graphgen.sample_sources(mask, 6, seed=1)
    for _ in range(6):
        g.set_options(schedule=4, schedule_mask=int(rng.integers(0, 2**63)), td_parent=int(rng.integers(0, 2)))
        check_against_oracle(og, g, sources, stats=True, th=16)


@pytest.fixture(scope="module")
def rmat16():
    scale = 16
    src, dst = graphgen.rmat_host(scale, seed=16)
    n = 1 << scale
    og = oracle.Graph(n, src, dst)
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    sources = graphgen.sample_sources(mask, 64, seed=1601)
    return n, src, dst, og, sources


def test_rmat16_topdown_64_sources(rmat16):
    """RMAT scale 16, plain top-down BFS, 64 seeded sources: bit-exact."""
    n, src, dst, og, sources = rmat16
    g = gpu_graph(n, src, dst, th=64, schedule=1)
    check_against_oracle(og, g, sources, stats=True, th=64)


@pytest.mark.parametrize("th", [0, 32, 64, 128, 256, 10**9])
def test_rmat16_direction_optimized_th(rmat16, th):
    n, src, dst, og, sources = rmat16
    g = gpu_graph(n, src, dst, th=th, device_edges=True)
    check_against_oracle(og, g, sources[:16], stats=True, th=th)
    g.set_options(schedule=5)
    check_against_oracle(og, g, sources[16:24], stats=True, th=th)
    g.set_options(td_parent=1)
    check_against_oracle(og, g, sources[24:32], stats=True, th=th)


def test_builder_layout_matches_oracle(rmat16):
    """Degree separation and renumbering (Sec. III-A, Fig. 2), rows sorted by caller id."""
    n, src, dst, og, _ = rmat16
    for th in (0, 16, 64, 10**9):
        g = gpu_graph(n, src, dst, th=th)
        off, col, co, io = g.export()
        want_io, want_co, d, n_ni = og.separate(th)
        assert g.info.delegates == d and g.info.n_nonisolated == n_ni
        assert_same(io, want_io, "internal_of")
        assert_same(co, want_co, "caller_of")
        ooff, ocol = og.csr()
        deg = np.diff(ooff)
        assert_same(np.diff(off), deg[co[:n_ni]], "degrees")
        # every internal row, mapped back to caller ids, equals the oracle row
        rows = co[col]
        for v in range(0, n_ni, 97):
            c = co[v]
            assert_same(rows[off[v]:off[v + 1]], ocol[ooff[c]:ooff[c + 1]], "row %d" % c)
        assert g.info.nnz == og.nnz
        assert list(g.info.subgraph_edges) == list(og.subgraph_counts(th))
        assert g.info.max_degree == deg.max()


def test_fig2_delegates_on_device():
    from tests.golden_io import read_fig2

    th, n, delegates, src, dst = read_fig2()
    g = gpu_graph(n, src, dst, th=th)
    _, _, co, io = g.export()
    assert g.info.delegates == len(delegates)
    for v, want in delegates.items():
        assert io[v] == want and co[want] == v


def test_host_output_buffers_match_device(rmat16):
    """Runs with host result buffers (copies inside the call) give the same output."""
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    n, src, dst, og, sources = rmat16
    g = gpu_graph(n, src, dst, th=64)
    hd = torch.empty(n, dtype=torch.int32).pin_memory()
    hp = torch.empty(n, dtype=torch.int32).pin_memory()
    for s in sources[:4]:
        bfs.bfs_run(g.handle, int(s), hd, hp)
        d, p = gpu_bfs(g, int(s))
        assert_same(hd.numpy(), d, "depth")
        assert_same(hp.numpy(), p, "parent")
    nd = np.empty(n, np.int32)
    npar = np.empty(n, np.int32)
    bfs.bfs_run(g.handle, int(sources[5]), nd, npar)
    want_d, want_p = og.bfs(int(sources[5]))
    assert_same(nd, want_d, "depth")
    assert_same(npar, want_p, "parent")


def test_repeated_runs_and_streams(rmat16):
    torch = need_cuda()
    n, src, dst, og, sources = rmat16
    g = gpu_graph(n, src, dst, th=32)
    st = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(st):
        for s in sources[:8]:
            d = torch.empty(n, dtype=torch.int32, device="cuda")
            p = torch.empty(n, dtype=torch.int32, device="cuda")
            g.run(int(s), d, p, stream=st)
            outs.append((int(s), d, p))
    g.wait(st)
    for s, d, p in outs:
        want_d, want_p = og.bfs(s)
        assert_same(d.cpu().numpy(), want_d, "depth")
        assert_same(p.cpu().numpy(), want_p, "parent")


def test_pinned_host_buffers_match_oracle():
    """Page-locked host result buffers are written by the kernel directly (no device
    copy); the results are the oracle's, for the single-source and batched calls."""
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    scale = 14
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=214)
    og = oracle.Graph(n, src, dst)
    g = gpu_graph(n, src, dst, th=32)
    mask = (np.diff(og.csr()[0]) > 0).astype(np.uint8)
    sources = graphgen.sample_sources(mask, 6, seed=2141)
    hd = torch.empty(n, dtype=torch.int32).pin_memory()
    hp = torch.empty(n, dtype=torch.int32).pin_memory()
    for s in sources:
        want_d, want_p = og.bfs(int(s))
        hd.fill_(7)
        hp.fill_(7)
        bfs.bfs_run(g.handle, int(s), hd, hp)
        assert_same(hd.numpy(), want_d, "pinned depth (source %d)" % s)
        assert_same(hp.numpy(), want_p, "pinned parent (source %d)" % s)
    b = bfs.Batch(g)
    bd = torch.empty((len(sources), n), dtype=torch.uint8).pin_memory()
    bp = torch.empty((len(sources), n), dtype=torch.int32).pin_memory()
    bfs.bfs_run_batch(b._h, sources, bd, bp)
    want_d, want_p = og.bfs_batch_u8(sources)
    for j in range(len(sources)):
        assert_same(bd[j].numpy(), want_d[j], "pinned batch depth %d" % j)
        assert_same(bp[j].numpy(), want_p[j], "pinned batch parent %d" % j)
    b.close()


@pytest.mark.parametrize("bps", [1, 3])
def test_other_level_loop_builds_match_oracle(rmat16, bps):
    """The 1024-thread (one CTA per SM) and 40-register (three per SM) builds of
    the level loop give the oracle's results, counters included."""
    n, src, dst, og, sources = rmat16
    g = gpu_graph(n, src, dst, th=64, blocks_per_sm=bps)
    check_against_oracle(og, g, sources[:16], stats=True, th=64)
    for sched in ("bottomup", "alternate"):
        g.set_options(**SCHEDULES[sched])
        check_against_oracle(og, g, sources[:4])
    g.close()


def test_depth_invariant_under_relabeling():
    """Metamorphic: relabelling the vertices by a permutation pi leaves every hop
    distance unchanged (depth'[pi(v)] = depth[v] from pi(s)); the parent is not
    invariant (the canonical pick is by id), but it is the oracle's either way."""
    need_cuda()
    scale = 13
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=313)
    perm = np.random.default_rng(313).permutation(n).astype(np.int32)
    og = oracle.Graph(n, src, dst)
    og2 = oracle.Graph(n, perm[src], perm[dst])
    g = gpu_graph(n, src, dst, th=32)
    g2 = gpu_graph(n, perm[src], perm[dst], th=32)
    mask = (np.diff(og.csr()[0]) > 0).astype(np.uint8)
    for s in graphgen.sample_sources(mask, 8, seed=3131):
        d, p = gpu_bfs(g, int(s))
        d2, p2 = gpu_bfs(g2, int(perm[s]))
        assert_same(d2[perm], d, "depth after relabelling (source %d)" % s)
        assert_same(p2, og2.bfs(int(perm[s]))[1], "parent of the relabelled graph (source %d)" % s)


@pytest.mark.parametrize("th", [5, 6, 7])
def test_degree_exactly_th(th):
    """A vertex of degree exactly TH stays normal, TH + 1 makes it a delegate
    (strictly greater, Sec. III-A); results are the oracle's either way."""
    need_cuda()
    # hub 0 of degree 6 and hub 7 of degree 7 in a graph of 40 vertices
    e = [(0, x) for x in range(1, 7)] + [(7, x) for x in range(8, 15)] + [(6, 8), (14, 20), (20, 21)]
    e = np.asarray(e, np.int32)
    n = 40
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th)
    want_d = int(og.separate(th)[2])
    assert g.info.delegates == want_d == (2 if th < 6 else (1 if th == 6 else 0))
    for s in (0, 3, 7, 21, 30):
        check_against_oracle(og, g, [s], stats=True, th=th)


@pytest.mark.parametrize("th", [16, 4000])
def test_long_row_drain(th):
    """Backward levels hand rows that settle nothing in their first entries to a
    list drained by all warps: hub 0 (leaves 1..10000) finds its only frontier
    neighbour at row position 9998, past the short-row group scan; results and
    counters are the oracle's (forced backward from level 1)."""
    need_cuda()
    n_leaf = 10000
    e = [(0, x) for x in range(1, n_leaf + 1)] + [(n_leaf + 1, n_leaf - 1), (n_leaf + 2, 5)]
    e = np.asarray(e, np.int32)
    n = n_leaf + 10
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th, schedule=2)
    check_against_oracle(og, g, [n_leaf + 1, n_leaf + 2, 0, 7], stats=True, th=th)


@pytest.mark.parametrize("th", [16, 4000])
@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_group_scan_hit_positions(th, shift):
    """A backward scan past the head entries reads a short row in aligned 4-entry
    loads: the hub's only frontier neighbour sits at every position class of the
    row (head, the first masked load, 4-entry and 16-entry boundaries, the last
    entry), and `shift` extra entries in a lower row move the hub's row start off
    the 4-entry grid (with TH 4000 the hub is a normal vertex and keeps its place).
    Depth, parent and the examined-entry counters equal the oracle's."""
    need_cuda()
    n_leaf, hub = 70, 10
    leaves = list(range(hub + 1, hub + 1 + n_leaf))
    e = [(hub, x) for x in leaves] + [(i, leaves[-1]) for i in range(shift)]
    positions = [0, 1, 3, 4, 5, 6, 7, 8, 15, 16, 19, 20, 21, 35, 36, 52, n_leaf - 1]
    sources = []
    for j, pos in enumerate(positions):
        s_j = hub + 1 + n_leaf + j
        e.append((s_j, leaves[pos]))
        sources.append(s_j)
    e = np.asarray(e, np.int32)
    n = hub + 1 + n_leaf + len(positions)
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th, schedule=2)
    check_against_oracle(og, g, sources, stats=True, th=th)


@pytest.mark.parametrize("th", [16, 10**9])
def test_first_level_from_source_row(th):
    """Level 0 runs straight from the source's row: a centre with 3000 leaves (six
    delegate chunks, or a normal row with TH 10^9) and a leaf whose only
    neighbour is that centre, in every schedule and both parent options; a
    few leaf-leaf edges give level 1 visited neighbours.  Depth, parent and the
    per-level counters equal the oracle's."""
    need_cuda()
    n_leaf = 3000
    e = [(0, x) for x in range(1, n_leaf + 1)] + [(x, x + 1) for x in range(1, 40, 2)]
    e += [(n_leaf + 1, n_leaf + 2), (n_leaf + 2, 0)]
    e = np.asarray(e, np.int32)
    n = n_leaf + 5
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th)
    for sched, opts in SCHEDULES.items():
        for tdp in (0, 1):
            g.set_options(td_parent=tdp, **opts)
            check_against_oracle(og, g, [0, 7, n_leaf, n_leaf + 1, n_leaf + 4], stats=True, th=th)


@pytest.mark.parametrize("sched", ["beamer", "topdown", "bottomup", "alternate"])
def test_deep_paths_all_depth_nibbles(sched):
    """Depths well past 15, 255 and 4095 (the depth is kept in 4-bit nibbles, a
    plane of them per 4 bits): a path of 4200 vertices with a pendant star and a
    ragged vertex count, from an end, from the middle and from a star leaf;
    then a short run on the same graph, so that nibbles a deep run left behind
    must not leak into the next result."""
    n = 4200 + 45
    e = [(i, i + 1) for i in range(4199)] + [(4199, 4200 + k) for k in range(45)]
    e = np.asarray(e, dtype=np.int32)
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=8, **SCHEDULES[sched])
    for s in (0, 2100, 4230, 4199):
        want_d, want_p = og.bfs(s)
        d, p = gpu_bfs(g, s)
        assert_same(d, want_d, "depth (source %d)" % s)
        assert_same(p, want_p, "parent (source %d)" % s)
    g.close()
