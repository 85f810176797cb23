"""Batched form (64-lane bitset multi-source BFS) vs the oracle's uint8 batched
BFS, bit-exact: depth (255 = unreached) and canonical parent for every query."""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from tests.gpu_util import assert_same, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def _batch_check(og, g, sources, with_parents=True, host=False):
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    b = bfs.Batch(g, with_parents=with_parents)
    want_d, want_p = og.bfs_batch_u8(sources)
    if host:
        k, n = len(sources), g.n
        d = np.empty((k, n), np.uint8)
        p = np.empty((k, n), np.int32) if with_parents else None
        bfs.bfs_run_batch(b._h, sources, d, p)
    else:
        d, p, st = b.run(sources, stats=True)
        d = d.cpu().numpy()
        p = p.cpu().numpy() if with_parents else None
        assert st.pairs_reached == int((want_d != 255).sum()) - sum(
            1 for s in sources if True)  # every source lane reaches its source at depth 0
    for j, s in enumerate(sources):
        assert_same(d[j], want_d[j], "depth of query %d (source %d)" % (j, s))
        if with_parents:
            assert_same(p[j], want_p[j], "parent of query %d (source %d)" % (j, s))
    b.close()


def _closed():
    R, C = 9, 13
    grid = []
    for r in range(R):
        for c in range(C):
            if r + 1 < R:
                grid.append((r * C + c, (r + 1) * C + c))
            if c + 1 < C:
                grid.append((r * C + c + 1, r * C + c))
    return {
        "path": (50, [(i, i + 1) for i in range(49)]),
        "star": (70, [(13, v) for v in range(70) if v != 13]),
        "grid": (R * C, grid),
        "cycle": (66, [(i, (i + 1) % 66) for i in range(66)]),
        "complete": (30, list(itertools.combinations(range(30), 2))),
        "components": (75, [(0, 1), (1, 2), (40, 41), (41, 42), (42, 43), (70, 71)]),
    }


@pytest.mark.parametrize("name", list(_closed().keys()))
@pytest.mark.parametrize("th", [0, 3, 64])
def test_batch_closed_forms(name, th):
    n, e = _closed()[name]
    e = np.asarray(e, np.int32)
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th)
    rng = np.random.default_rng(n + th)
    sources = rng.integers(0, n, 64)
    _batch_check(og, g, sources)
    _batch_check(og, g, sources[:5])  # a partial batch
    _batch_check(og, g, [int(sources[0])] * 3 + [n - 1])  # repeated sources


def test_batch_random_graphs():
    rng = np.random.default_rng(77)
    for trial in range(20):
        n = int(rng.integers(2, 600))
        m = int(rng.integers(0, 8 * n))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        og = oracle.Graph(n, src, dst)
        g = gpu_graph(n, src, dst, th=int(rng.choice([0, 4, 16, 10**9])))
        k = int(rng.integers(1, 65))
        _batch_check(og, g, rng.integers(0, n, k), with_parents=bool(trial % 4))


def test_batch_rmat16_64_sources():
    scale = 16
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=16)
    og = oracle.Graph(n, src, dst)
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    sources = graphgen.sample_sources(mask, 64, seed=1601)
    for th in (0, 64, 10**9):
        g = gpu_graph(n, src, dst, th=th)
        _batch_check(og, g, sources)
    _batch_check(og, g, sources[:33], host=True)


@pytest.mark.parametrize("ctas", [1, 37, 152])
def test_batch_grid_sizes(ctas):
    """A context may take any CTA count up to the co-resident capacity (the
    serving loop runs several such launches side by side)."""
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    scale = 14
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=14)
    og = oracle.Graph(n, src, dst)
    g = gpu_graph(n, src, dst, th=32)
    assert ctas <= bfs.bfs_batch_capacity()
    sources = np.random.default_rng(ctas).integers(0, n, 40)
    want_d, want_p = og.bfs_batch_u8(sources)
    b = bfs.Batch(g, ctas=ctas)
    for k in (1, 3, 40):  # lane strides 4, 4, 40
        d, p = b.run(sources[:k])
        for j in range(k):
            assert_same(d[j].cpu().numpy(), want_d[j], "depth, %d CTAs, lane %d of %d" % (ctas, j, k))
            assert_same(p[j].cpu().numpy(), want_p[j], "parent, %d CTAs, lane %d of %d" % (ctas, j, k))
    with pytest.raises(bfs.BfsError):
        bfs.Batch(g, ctas=bfs.bfs_batch_capacity() + 1)
    b.close()


@pytest.mark.parametrize("th", [16, 64])
def test_batch_deferred_long_rows(th):
    """Backward levels split a long row past its first 512 entries into chunks run
    by different warps: the canonical parent is then the smallest first hit over
    the chunks.  Hub 0 has leaves 1..3000 (its row in caller order); each query's
    source hangs off one or two leaves, so at level 1 the hub's only frontier
    neighbours sit inside the head, in one deferred chunk, or in two chunks."""
    need_cuda()
    import paper_1803_03922_gb300 as bfs

    n_leaf = 3000
    e = [(0, x) for x in range(1, n_leaf + 1)]
    attach = [[100], [700], [2000, 700], [2999], [1500, 2600], [513], [514, 1030], [3000, 5]]
    n = n_leaf + 1 + len(attach)
    for j, xs in enumerate(attach):
        e += [(n_leaf + 1 + j, x) for x in xs]
    e = np.asarray(e, np.int32)
    og = oracle.Graph(n, e[:, 0], e[:, 1])
    g = gpu_graph(n, e[:, 0], e[:, 1], th=th, alpha=1 << 30)  # backward from level 1 on
    sources = [n_leaf + 1 + j for j in range(len(attach))]
    _batch_check(og, g, sources)
    _, want_p = og.bfs_batch_u8(sources)
    assert [int(want_p[j][0]) for j in range(len(attach))] == [min(xs) for xs in attach]
    b = bfs.Batch(g)
    _, _, st = b.run(sources, stats=True)
    assert [st.level[i].direction for i in range(st.logged_levels)][:2] == [0, 1]
    b.close()


def test_batch_lanes_that_finish_early():
    """Lanes whose source lies in a small component run out of frontier after a
    few levels and are no longer searched for in backward levels; the other
    lanes' results are unchanged (backward from level 1 on)."""
    need_cuda()
    scale = 12
    n_big = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=312)
    extra = [(n_big + i, n_big + i + 1) for i in range(3)] + [(n_big + 10, n_big + 11)]
    e = np.asarray(extra, np.int32)
    src = np.concatenate([src, e[:, 0]]).astype(np.int32)
    dst = np.concatenate([dst, e[:, 1]]).astype(np.int32)
    n = n_big + 20
    og = oracle.Graph(n, src, dst)
    g = gpu_graph(n, src, dst, th=16, alpha=1 << 30)
    mask = (np.diff(og.csr()[0][: n_big + 1]) > 0).astype(np.uint8)
    big = graphgen.sample_sources(mask, 60, seed=3121)
    sources = list(big[:30]) + [n_big, n_big + 3, n_big + 10, n_big + 15] + list(big[30:])
    _batch_check(og, g, sources)


def test_batch_isolated_and_overflow():
    torch = need_cuda()
    import paper_1803_03922_gb300 as bfs

    e = np.array([(i, i + 1) for i in range(299)], np.int32)  # path: depth 299 from an end
    og = oracle.Graph(302, e[:, 0], e[:, 1])
    g = gpu_graph(302, e[:, 0], e[:, 1], th=8)
    _batch_check(og, g, [150, 301, 100])  # 301 is isolated; depths <= 200
    b = bfs.Batch(g)
    with pytest.raises(bfs.BfsError) as ex:
        b.run([150, 0], stats=True)
    assert ex.value.code == bfs.BFS_ERR_OVERFLOW
    d, p, st = b.run([150], stats=True)  # the context stays usable
    dn = d.cpu().numpy()
    assert int(dn[dn != 255].max()) == 150 and st.levels == 151
    d, p, st = b.run([301, 301], stats=True)  # isolated sources only: depth 0 is the deepest
    assert st.levels == 1 and st.logged_levels == 0 and st.pairs_reached == 0


def test_batch_order_groups_by_second_frontier():
    """bfs_batch_order returns a permutation sorted by the degree sum of each
    source's neighbours (computed here from the oracle's CSR), largest first,
    ties in input order; batches cut from it still equal the oracle."""
    need_cuda()
    import paper_1803_03922_gb300 as bfs

    scale = 14
    n = 1 << scale
    src, dst = graphgen.rmat_host(scale, seed=1414)
    og = oracle.Graph(n, src, dst)
    off, col = og.csr()[:2]
    deg = np.diff(off)
    key = lambda s: int(deg[col[off[s]:off[s + 1]]].sum())
    rng = np.random.default_rng(14)
    sources = rng.integers(0, n, 200)  # isolated sources and repeats included
    g = gpu_graph(n, src, dst, th=16)
    order = bfs.bfs_batch_order(g.handle, sources)
    assert sorted(order.tolist()) == list(range(len(sources)))
    want = sorted(range(len(sources)), key=lambda j: (-key(sources[j]), j))
    assert order.tolist() == want
    grouped = sources[order]
    for i in range(0, len(grouped), 64):
        _batch_check(og, g, grouped[i:i + 64])
    assert bfs.bfs_batch_order(g.handle, np.zeros(0, np.int32)).size == 0
    with pytest.raises(bfs.BfsError):
        bfs.bfs_batch_order(g.handle, np.array([n], np.int32))
