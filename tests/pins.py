"""Pins for the CPU oracle: checks against what the mathematics fixes, written
independently of ``oracle.c`` (closed forms, shortest-path enumeration,
library routines, invariants).  ``run_all(lib)`` runs every pin against a given
build of the oracle and returns the names of the pins that failed, so a test
can also show that a deliberately broken oracle is caught.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle


def _g(n, edges, lib):
    if len(edges):
        e = np.asarray(edges, dtype=np.int32)
        return oracle.Graph(n, e[:, 0], e[:, 1], lib=lib)
    return oracle.Graph(n, np.zeros(0, np.int32), np.zeros(0, np.int32), lib=lib)


# ---- closed forms -------------------------------------------------------------------------

def pin_path_end(lib):
    n = 37
    g = _g(n, [(i, i + 1) for i in range(n - 1)], lib)
    d, p = g.bfs(0)
    return (d == np.arange(n)).all() and p[0] == 0 and (p[1:] == np.arange(n - 1)).all()


def pin_path_middle(lib):
    n, s = 41, 17
    g = _g(n, [(i + 1, i) for i in range(n - 1)], lib)
    d, p = g.bfs(s)
    want_d = np.abs(np.arange(n) - s)
    want_p = np.where(np.arange(n) < s, np.arange(n) + 1, np.arange(n) - 1)
    want_p[s] = s
    return (d == want_d).all() and (p == want_p).all()


def pin_star(lib):
    n, c = 50, 13
    g = _g(n, [(c, v) for v in range(n) if v != c], lib)
    d, p = g.bfs(c)
    ok = d[c] == 0 and (np.delete(d, c) == 1).all() and (np.delete(p, c) == c).all() and p[c] == c
    leaf = 40
    d, p = g.bfs(leaf)
    want = np.full(n, 2)
    want[c], want[leaf] = 1, 0
    wp = np.full(n, c)
    wp[leaf] = leaf
    wp[c] = leaf
    return ok and (d == want).all() and (p == wp).all()


def pin_grid(lib):
    R, C = 9, 13
    ids = lambda r, c: r * C + c  # noqa: E731
    e = []
    for r in range(R):
        for c in range(C):
            if r + 1 < R:
                e.append((ids(r, c), ids(r + 1, c)))
            if c + 1 < C:
                e.append((ids(r, c + 1), ids(r, c)))
    g = _g(R * C, e, lib)
    d, p = g.bfs(0)
    for r in range(R):
        for c in range(C):
            v = ids(r, c)
            if d[v] != r + c:
                return False
            if v == 0:
                if p[v] != 0:
                    return False
                continue
            # the up-neighbour has the smaller row-major id whenever it exists
            want = ids(r - 1, c) if r > 0 else ids(r, c - 1)
            if p[v] != want:
                return False
    return True


def pin_binary_tree(lib):
    n = 255
    g = _g(n, [((i - 1) // 2, i) for i in range(1, n)], lib)
    d, p = g.bfs(0)
    i = np.arange(n)
    want_d = np.floor(np.log2(i + 1)).astype(np.int64)
    want_p = (i - 1) // 2
    want_p[0] = 0
    return (d == want_d).all() and (p == want_p).all()


def pin_complete(lib):
    n, s = 12, 5
    g = _g(n, list(itertools.combinations(range(n), 2)), lib)
    d, p = g.bfs(s)
    want_d = np.ones(n)
    want_d[s] = 0
    return (d == want_d).all() and (p == s).all() and g.nnz == n * (n - 1)


def pin_even_cycle(lib):
    n = 20
    g = _g(n, [(i, (i + 1) % n) for i in range(n)], lib)
    d, p = g.bfs(0)
    i = np.arange(n)
    want_d = np.minimum(i, n - i)
    want_p = np.where(i < n // 2, i - 1, (i + 1) % n)
    want_p[0] = 0
    want_p[n // 2] = n // 2 - 1  # antipode: two parents at the same depth, the smaller wins
    return (d == want_d).all() and (p == want_p).all()


def pin_components_and_isolated(lib):
    # two paths and an isolated vertex; source in the second path
    e = [(0, 1), (1, 2), (4, 5), (5, 6), (6, 7)]
    g = _g(9, e, lib)
    d, p = g.bfs(5)
    ok = list(d) == [-1, -1, -1, -1, 1, 0, 1, 2, -1] and list(p) == [-1, -1, -1, -1, 5, 5, 5, 6, -1]
    d, p = g.bfs(8)  # isolated source
    want = [-1] * 9
    want[8] = 0
    wp = [-1] * 9
    wp[8] = 8
    return ok and list(d) == want and list(p) == wp


def pin_dedup_selfloops(lib):
    e = [(0, 1), (1, 0), (0, 1), (2, 2), (1, 2), (2, 1), (3, 3)]
    g = _g(4, e, lib)
    off, col = g.csr()
    return list(off) == [0, 1, 3, 4, 4] and list(col) == [1, 0, 2, 1] and g.nnz == 4


# ---- brute force --------------------------------------------------------------------------

def _shortest_paths_enum(n, adj, s):
    """All simple paths from s, kept when shortest; returns (dist, min penultimate)."""
    dist = [-1] * n
    pen = [-1] * n
    dist[s] = 0
    pen[s] = s
    stack = [(s, (s,))]
    paths = {}
    while stack:
        v, path = stack.pop()
        for u in range(n):
            if adj[v][u] and u not in path:
                L = len(path)
                paths.setdefault(u, []).append((L, v))
                stack.append((u, path + (u,)))
    for u, lst in paths.items():
        L = min(x for x, _ in lst)
        dist[u] = L
        pen[u] = min(v for x, v in lst if x == L)
    return dist, pen


def pin_exhaustive_5(lib):
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        adj = [[0] * n for _ in range(n)]
        for a, b in e:
            adj[a][b] = adj[b][a] = 1
        g = _g(n, e, lib)
        for s in range(n):
            d, p = g.bfs(s)
            wd, wp = _shortest_paths_enum(n, adj, s)
            if list(d) != wd or list(p) != wp:
                return False
    return True


def pin_random_small_floyd(lib, trials=300, seed=1):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 11))
        m = int(rng.integers(0, 3 * n))
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        g = oracle.Graph(n, src, dst, lib=lib)
        A = np.zeros((n, n), dtype=bool)
        A[src, dst] = True
        A[dst, src] = True
        np.fill_diagonal(A, False)
        INF = 10**9
        D = np.where(A, 1, INF)
        np.fill_diagonal(D, 0)
        for k in range(n):  # Floyd-Warshall relaxation
            D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
        s = int(rng.integers(0, n))
        d, p = g.bfs(s)
        want_d = np.where(D[s] >= INF, -1, D[s])
        if not (d == want_d).all():
            return False
        adjl = A.astype(int).tolist()
        if n <= 8:
            _, wp = _shortest_paths_enum(n, adjl, s)
            if list(p) != wp:
                return False
    return True


# ---- library routines and invariants ------------------------------------------------------

def _random_graph(rng, n, m):
    return rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32)


def pin_scipy_depth_components(lib, seed=7):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components, shortest_path

    rng = np.random.default_rng(seed)
    n, m = 700, 900  # sparse: several components
    src, dst = _random_graph(rng, n, m)
    g = oracle.Graph(n, src, dst, lib=lib)
    A = sp.coo_matrix((np.ones(m), (src, dst)), shape=(n, n)).tocsr()
    A = ((A + A.T) > 0).astype(np.int8)
    A.setdiag(0)
    A.eliminate_zeros()
    _, lab = connected_components(A, directed=False)
    for s in rng.integers(0, n, 6):
        d, p = g.bfs(int(s))
        ref = shortest_path(A, method="D", unweighted=True, indices=int(s))
        want = np.where(np.isinf(ref), -1, ref).astype(np.int64)
        if not (d == want).all():
            return False
        if not ((d >= 0) == (lab == lab[s])).all():
            return False
    return True


def pin_invariants_python(lib, seed=11):
    """Graph500-style rules checked by code independent of the oracle's validator."""
    rng = np.random.default_rng(seed)
    n, m = 400, 1500
    src, dst = _random_graph(rng, n, m)
    g = oracle.Graph(n, src, dst, lib=lib)
    off, col = g.csr()
    for s in rng.integers(0, n, 5):
        s = int(s)
        d, p = g.bfs(s)
        if d[s] != 0 or p[s] != s:
            return False
        for u in range(n):
            nb = col[off[u]:off[u + 1]]
            if ((d[u] >= 0) != (d[nb] >= 0)).any():
                return False
            if d[u] >= 0 and (np.abs(d[u] - d[nb]) > 1).any():
                return False
            if u == s:
                continue
            if d[u] < 0:
                if p[u] != -1:
                    return False
                continue
            cands = nb[d[nb] == d[u] - 1]
            if p[u] not in set(nb.tolist()) or p[u] != cands.min():
                return False
    return True


def pin_validator_detects(lib):
    """The validator accepts the oracle's own answer and rejects planted faults."""
    e = [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (5, 6)]
    g = _g(7, e, lib)
    d, p = g.bfs(0)
    if g.validate(0, d, p) != 0:
        return False
    checks = []
    p2 = p.copy(); p2[3] = 2; checks.append((d, p2, 6))          # non-canonical parent
    p2 = p.copy(); p2[4] = 0; checks.append((d, p2, 4))          # parent is not a neighbour
    d2 = d.copy(); d2[4] = 5; checks.append((d2, p, 3))          # depth jump on an edge
    d2 = d.copy(); d2[4] = -1; p2 = p.copy(); p2[4] = -1; checks.append((d2, p2, 2))
    d2 = d.copy(); d2[0] = 1; checks.append((d2, p, 1))
    p2 = p.copy(); p2[5] = 6; checks.append((d, p2, 7))
    p2 = p.copy(); p2[1] = 3; checks.append((d, p2, 5))          # parent is a neighbour one level deeper
    p2 = p.copy(); p2[3] = 4; checks.append((d, p2, 5))          # parent is a neighbour one level deeper
    # Rule 8 (reached set = component of s) follows from rules 1-7: a parent chain
    # falls one level per step, so it ends at the only vertex of depth 0, s, and
    # no edge leaves the reached set.  A wrong union-find (a mutant) is caught by
    # the oracle's own answer being rejected above.
    return all(g.validate(0, a, b) == want for a, b, want in checks)


def pin_component_edges(lib, seed=3):
    rng = np.random.default_rng(seed)
    n, m = 300, 500
    src, dst = _random_graph(rng, n, m)
    g = oracle.Graph(n, src, dst, lib=lib)
    s = int(src[0])
    d, _ = g.bfs(s)
    pairs = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist()) if a != b}
    want = sum(1 for a, b in pairs if d[a] >= 0)
    return g.component_edges(d) == want


def pin_builder_sets(lib, seed=5):
    rng = np.random.default_rng(seed)
    for n, m in [(1, 3), (17, 60), (200, 3000)]:
        src, dst = _random_graph(rng, n, m)
        g = oracle.Graph(n, src, dst, lib=lib)
        off, col = g.csr()
        rows = [set() for _ in range(n)]
        for a, b in zip(src.tolist(), dst.tolist()):
            if a != b:
                rows[a].add(b)
                rows[b].add(a)
        for u in range(n):
            if col[off[u]:off[u + 1]].tolist() != sorted(rows[u]):
                return False
    return True


def pin_separation(lib, seed=9):
    """Sec. III-A: delegate iff degree > TH, delegate ids ascending (Fig. 2), then
    non-isolated normal vertices, then isolated ones, each ascending."""
    rng = np.random.default_rng(seed)
    n, m = 500, 2500
    src, dst = _random_graph(rng, n, m)
    src[:40] = 3  # a hub
    g = oracle.Graph(n, src, dst, lib=lib)
    deg = g.degree()
    for th in [-1, 0, 5, int(np.median(deg)), int(deg.max()) - 1, int(deg.max())]:
        io, co, d, n_ni = g.separate(th)
        dl = np.flatnonzero(deg > th)
        nl = np.flatnonzero((deg > 0) & (deg <= th))
        il = np.flatnonzero((deg == 0) & (deg <= th))
        if th < 0:
            nl = np.zeros(0, dtype=np.int64)
            il = np.zeros(0, dtype=np.int64)
        order = np.concatenate([dl, nl, il])
        if d != dl.size or n_ni != dl.size + nl.size:
            return False
        if not (co == order).all() or not (io[order] == np.arange(n)).all():
            return False
    return True


def pin_subgraph_counts(lib, seed=13):
    rng = np.random.default_rng(seed)
    n, m = 300, 2000
    src, dst = _random_graph(rng, n, m)
    src[:50] = 7
    g = oracle.Graph(n, src, dst, lib=lib)
    off, col = g.csr()
    deg = np.diff(off)
    for th in [0, 4, 8, 16, 10**9]:
        got = g.subgraph_counts(th)
        want = np.zeros(4, dtype=np.int64)
        for u in range(n):
            for v in col[off[u]:off[u + 1]]:
                want[2 * int(deg[u] > th) + int(deg[v] > th)] += 1
        if not (got == want).all() or got.sum() != g.nnz or got[1] != got[2]:
            return False
    return True


def pin_batch_u8(lib):
    e = [(i, i + 1) for i in range(30)] + [(40, 41)]
    g = _g(50, e, lib)
    srcs = [0, 15, 40, 45]
    D, P = g.bfs_batch_u8(srcs)
    for j, s in enumerate(srcs):
        d, p = g.bfs(s)
        if not (D[j] == np.where(d < 0, 255, d)).all() or not (P[j] == p).all():
            return False
    # a path of 300 vertices from an end reaches depth 299 > 254
    g2 = _g(300, [(i, i + 1) for i in range(299)], lib)
    try:
        g2.bfs_batch_u8([0])
        return False
    except OverflowError:
        pass
    D, _ = g2.bfs_batch_u8([150])  # depth <= 150 fits
    return int(D.max()) == 150


def pin_level_counters_closed_forms(lib):
    """Path 0-1-...-(n-1) from vertex 0, every level backward: at level L the
    unvisited vertices are L+1..n-1; L+1 finds L at its first entry, every later
    vertex reads its whole row (degree 2, the last one degree 1)."""
    n = 12
    g = _g(n, [(i, i + 1) for i in range(n - 1)], lib)
    d, _ = g.bfs(0)
    levels = n
    dirs = np.ones(levels, dtype=np.int32)
    c = g.level_counters(0, d, 64, dirs)
    for L in range(levels):
        unv = list(range(L + 1, n))
        want_edges = sum(1 if v == L + 1 else (1 if v == n - 1 else 2) for v in unv)
        want = [1, 1 if L in (0, n - 1) else 2, 1 if L + 1 < n else 0, len(unv), want_edges, 0, 0]
        if list(c[L]) != want:
            return False
    # star from the centre, forward: level 0 frontier {c} (a normal vertex only if
    # its degree <= th), all leaves found, each leaf's only neighbour is c
    m = 9
    g = _g(m, [(0, v) for v in range(1, m)], lib)
    d, _ = g.bfs(0)
    c = g.level_counters(0, d, 4, np.array([0, 0], np.int32))
    ok = list(c[0]) == [1, m - 1, m - 1, 0, 0, m - 1, 0] and list(c[1]) == [m - 1, m - 1, 0, 0, 0, 0, m - 1]
    c2 = g.level_counters(0, d, 100, np.array([0, 1], np.int32))
    return ok and c2[0][6] == 1 and list(c2[1][3:5]) == [0, 0]


def pin_level_counters_first_hit(lib):
    """Column 5 (forward parent pick: first-hit position + 1 in the sorted row)
    and column 4 (backward k_v) where the first visited neighbour is not the
    first entry.  Edges 0-4, 0-5, 5-6, 1-6, 2-6, 3-6 from source 0: depth 1 =
    {4, 5}, depth 2 = {6}, depth 3 = {1, 2, 3}.  Row of 6 = [1, 2, 3, 5]: its
    parent 5 is the fourth entry.  Forward everywhere: level 0 picks for 4 ([0])
    and 5 ([0, 6]) one entry each = 2; level 1 picks for 6 = 4; level 2 picks
    for 1, 2, 3 (rows [6]) = 3.  Level 1 backward: the unvisited non-isolated
    vertices at its start are 1, 2, 3 (row [6], 6 unvisited: k = 1 each) and 6
    (k = 4): scanned 4, sum of k = 7."""
    g = _g(7, [(0, 4), (0, 5), (5, 6), (1, 6), (2, 6), (3, 6)], lib)
    d, _ = g.bfs(0)
    if d.tolist() != [0, 3, 3, 3, 1, 1, 2]:
        return False
    c = g.level_counters(0, d, 64, np.zeros(4, np.int32))
    if [int(c[L][5]) for L in range(4)] != [2, 4, 3, 0]:
        return False
    c = g.level_counters(0, d, 64, np.array([0, 1, 0, 0], np.int32))
    return list(c[1][3:5]) == [4, 7] and int(c[1][5]) == 0


def pin_directions_worked(lib):
    """The direction rules against the hand-worked levels of
    tests/golden/directions_worked.txt (Sec. IV-B)."""
    from tests.golden_io import read_directions

    graphs, cases = read_directions()
    built = {k: oracle.Graph(n, s, d, lib=lib) for k, (n, s, d) in graphs.items()}
    for gname, src, rule, a, b, want in cases:
        g = built[gname]
        d, _ = g.bfs(src)
        if rule == "paper":
            got = g.directions(src, d, "paper", factor0=a, factor1=b)
        else:
            got = g.directions(src, d, rule, alpha=int(a), beta=int(b))
        if list(got) != want:
            return False
    return True


def pin_subgraph_directions_worked(lib):
    """The per-subgraph rule against the hand-worked levels of
    tests/golden/subgraph_directions_worked.txt (Sec. IV-B)."""
    from tests.golden_io import read_subgraph_directions

    graphs, cases = read_subgraph_directions()
    for gname, src, f0, f1, want in cases:
        n, th, s, d = graphs[gname]
        g = oracle.Graph(n, s, d, lib=lib)
        dep, _ = g.bfs(src)
        if list(g.subgraph_directions(src, dep, th, f0, f1)) != want:
            return False
    return True


def pin_subgraph_directions_reduce(lib, seed=23):
    """Limit cases of the per-subgraph rule on random graphs: factor0 = 0 turns
    every subgraph backward at its first level with a frontier (FV > 0 = 0 BV);
    factor0 = infinity keeps all forward; with th at least the maximum degree
    there are no delegates, so dd, dn and nd never have a frontier and stay
    forward; with th = 0 every non-isolated vertex is a delegate, so only dd
    has work, and its decisions follow the single paper rule (Sec. IV-B) with
    U = s = the unvisited non-isolated vertices."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        n = int(rng.integers(5, 60))
        m = int(rng.integers(n, 4 * n))
        src, dst = _random_graph(rng, n, m)
        g = oracle.Graph(n, src, dst, lib=lib)
        s = int(src[0])
        d, _ = g.bfs(s)
        inf = float("inf")
        if g.subgraph_directions(s, d, 2, (inf,) * 3, (0.0,) * 3).any():
            return False
        big = int(g.degree().max())
        if g.subgraph_directions(s, d, big, (0.0,) * 3, (0.0,) * 3).any():
            return False
        for f0 in (0.05, 0.5, 2.0):
            dd = g.subgraph_directions(s, d, 0, (f0, 0.5, 0.5), (1e-7, 1e-7, 1e-7))
            one = g.directions(s, d, "paper", factor0=f0, factor1=1e-7)
            if list(dd & 1) != list(one) or (dd & 6).any():
                return False
        allb = g.subgraph_directions(s, d, 2, (0.0,) * 3, (0.0,) * 3)
        # a subgraph turns backward for good at the first level where it has a frontier
        if not np.all(np.diff(allb & 1) >= 0) or not np.all(np.diff((allb >> 1) & 1) >= 0):
            return False
    return True


def pin_directions_limits(lib, seed=17):
    """Limit cases of the rules on random graphs: factor0 = 0 goes backward at
    level 0 and (factor1 = 0) never returns; factor0 = inf or alpha = 0 never
    leaves forward; lowering factor0 or raising alpha never delays the first
    backward level."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        n = int(rng.integers(2, 80))
        e = rng.integers(0, n, (int(rng.integers(1, 4 * n)), 2)).astype(np.int32)
        g = oracle.Graph(n, e[:, 0], e[:, 1], lib=lib)
        s = int(e[0, 0]) if e[0, 0] != e[0, 1] else int(rng.integers(0, n))
        d, _ = g.bfs(s)
        levels = int(d.max()) + 1 if (g.csr()[0][s + 1] > g.csr()[0][s]) else 0
        if levels == 0:
            continue
        if list(g.directions(s, d, "paper", factor0=0.0, factor1=0.0)) != [1] * levels:
            return False
        if list(g.directions(s, d, "paper", factor0=float("inf"), factor1=0.0)) != [0] * levels:
            return False
        if list(g.directions(s, d, "beamer", alpha=0, beta=18)) != [0] * levels:
            return False

        def first_b(x):
            x = list(x)
            return x.index(1) if 1 in x else levels

        fp = [first_b(g.directions(s, d, "paper", factor0=f, factor1=0.0)) for f in (4.0, 1.0, 0.5, 0.1, 0.01)]
        fb = [first_b(g.directions(s, d, "beamer", alpha=a, beta=18)) for a in (1, 4, 15, 60, 1000)]
        if fp != sorted(fp, reverse=True) or fb != sorted(fb, reverse=True):
            return False
    return True


PINS = [
    pin_path_end, pin_path_middle, pin_star, pin_grid, pin_binary_tree, pin_complete,
    pin_even_cycle, pin_components_and_isolated, pin_dedup_selfloops, pin_exhaustive_5,
    pin_random_small_floyd, pin_scipy_depth_components, pin_invariants_python,
    pin_validator_detects, pin_component_edges, pin_builder_sets, pin_separation,
    pin_subgraph_counts, pin_batch_u8, pin_level_counters_closed_forms, pin_level_counters_first_hit,
    pin_directions_worked, pin_directions_limits, pin_subgraph_directions_worked,
    pin_subgraph_directions_reduce,
]


def run_all(lib, pins=None):
    failed = []
    for pin in pins or PINS:
        try:
            ok = bool(pin(lib))
        except Exception:  # a crash or a rejected call counts as a failed pin
            ok = False
        if not ok:
            failed.append(pin.__name__)
    return failed
