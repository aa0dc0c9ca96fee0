"""Pins for the oracle's BFS, CC and SSSP against things other than itself:
brute force on tiny graphs, SciPy's graph routines, and the invariants the
definitions fix (Section 5, "Applications")."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import graphgen as gg
import oracle

INF = oracle.INF


def _adj(g, weights=None):
    dst = g.dst()
    data = np.ones(g.E) if weights is None else weights.astype(np.float64)
    return sp.csr_matrix((data, (g.src.astype(np.int64), dst.astype(np.int64))), shape=(g.V, g.V))


def _floyd(g, w=None):
    """All-pairs shortest paths by plain triple loop (tiny graphs only)."""
    V = g.V
    D = [[float("inf")] * V for _ in range(V)]
    for i in range(V):
        D[i][i] = 0.0
    dst = g.dst()
    for p in range(g.E):
        u, v = int(g.src[p]), int(dst[p])
        c = 1.0 if w is None else float(w[p])
        D[u][v] = min(D[u][v], c)
    for k in range(V):
        Dk = D[k]
        for i in range(V):
            dik = D[i][k]
            if dik == float("inf"):
                continue
            Di = D[i]
            for j in range(V):
                if dik + Dk[j] < Di[j]:
                    Di[j] = dik + Dk[j]
    return D


def _as_u32(row):
    return np.array([INF if x == float("inf") else int(x) for x in row], dtype=np.uint32)


@pytest.mark.parametrize("seed", range(6))
def test_bfs_brute_force_tiny(seed):
    V = 12 + 5 * seed
    g = gg.random_graph(V, 2 * V, seed=100 + seed)
    D = _floyd(g)
    for root in (0, V // 2, V - 1):
        want = _as_u32(D[root])
        np.testing.assert_array_equal(oracle.bfs_push(g, root), want)
        np.testing.assert_array_equal(oracle.bfs_pull(g, root), want)


def test_bfs_matches_scipy_and_invariants():
    g = gg.rmat(11, 8)
    dist = csg.shortest_path(_adj(g), method="D", unweighted=True, directed=True, indices=0)
    want = np.where(np.isinf(dist), INF, dist).astype(np.uint32)
    push, pull = oracle.bfs_push(g, 0), oracle.bfs_pull(g, 0)
    np.testing.assert_array_equal(push, want)
    np.testing.assert_array_equal(pull, want)
    # level[v] <= level[u] + 1 on every edge u->v; every reached v != root
    # has an in-neighbour exactly one level up
    src, dst = g.src.astype(np.int64), g.dst().astype(np.int64)
    lu, lv = pull[src].astype(np.int64), pull[dst].astype(np.int64)
    reached_u = lu != INF
    assert np.all(lv[reached_u] <= lu[reached_u] + 1)
    parent_ok = np.zeros(g.V, dtype=bool)
    parent_ok[dst[(lv != INF) & (lu == lv - 1)]] = True
    reached = np.flatnonzero(pull != INF)
    assert np.all(parent_ok[reached[reached != 0]])


def test_bfs_undirected_grid_levels_differ_by_at_most_one():
    g = gg.grid(24, 0.05)
    lvl = oracle.bfs_pull(g, 0).astype(np.int64)
    src, dst = g.src.astype(np.int64), g.dst().astype(np.int64)
    assert np.all(np.abs(lvl[src] - lvl[dst]) <= 1)
    # plain grid: level is the Manhattan distance from the corner
    g0 = gg.grid(17, 0.0)
    lvl0 = oracle.bfs_push(g0, 0)
    r, c = np.divmod(np.arange(g0.V), 17)
    np.testing.assert_array_equal(lvl0, (r + c).astype(np.uint32))


def _cc_dfs(g):
    """Components by explicit DFS over the undirected adjacency (tiny graphs)."""
    nbr = [set() for _ in range(g.V)]
    dst = g.dst()
    for p in range(g.E):
        u, v = int(g.src[p]), int(dst[p])
        nbr[u].add(v)
        nbr[v].add(u)
    lab = [-1] * g.V
    for s in range(g.V):
        if lab[s] >= 0:
            continue
        stack, comp = [s], []
        lab[s] = s
        while stack:
            x = stack.pop()
            comp.append(x)
            for y in nbr[x]:
                if lab[y] < 0:
                    lab[y] = s
                    stack.append(y)
    return np.array(lab, dtype=np.uint32)  # s is the smallest id: visited in order


@pytest.mark.parametrize("seed", range(5))
def test_cc_brute_force_tiny(seed):
    V = 30 + 7 * seed
    g = gg.symmetrize(gg.random_graph(V, V // 2 + seed, seed=200 + seed))
    want = _cc_dfs(g)
    np.testing.assert_array_equal(oracle.cc_union_find(g), want)
    np.testing.assert_array_equal(oracle.cc_pull(g), want)


def test_cc_matches_scipy():
    g = gg.symmetrize(gg.rmat(12, 4))
    n, comp = csg.connected_components(_adj(g), directed=False)
    minid = np.full(n, np.iinfo(np.int64).max)
    np.minimum.at(minid, comp, np.arange(g.V))
    want = minid[comp].astype(np.uint32)
    np.testing.assert_array_equal(oracle.cc_union_find(g), want)
    np.testing.assert_array_equal(oracle.cc_pull(g), want)
    assert n > 1  # the R-MAT graph has isolated vertices: a non-trivial case


@pytest.mark.parametrize("seed", range(5))
def test_sssp_brute_force_tiny(seed):
    V = 10 + 6 * seed
    g = gg.random_graph(V, 3 * V, seed=300 + seed).with_weights(20, seed=seed)
    D = _floyd(g, g.w)
    for root in (0, V - 1):
        want = _as_u32(D[root])
        np.testing.assert_array_equal(oracle.sssp_dijkstra(g, root), want)
        np.testing.assert_array_equal(oracle.sssp_push(g, root), want)
        np.testing.assert_array_equal(oracle.sssp_pull(g, root), want)


def test_sssp_matches_scipy_triangle_and_tightness():
    g = gg.rmat(11, 8).with_weights(255)
    dist = csg.dijkstra(_adj(g, g.w), directed=True, indices=0)
    want = np.where(np.isinf(dist), INF, dist).astype(np.uint32)
    got = oracle.sssp_dijkstra(g, 0)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(oracle.sssp_pull(g, 0), want)
    src, dst = g.src.astype(np.int64), g.dst().astype(np.int64)
    du, dv, w = got[src].astype(np.int64), got[dst].astype(np.int64), g.w.astype(np.int64)
    fin = du != INF
    assert np.all(dv[fin] <= du[fin] + w[fin])          # triangle inequality
    tight = np.zeros(g.V, dtype=bool)
    tight[dst[fin & (dv == du + w)]] = True
    reached = np.flatnonzero(got != INF)
    assert np.all(tight[reached[reached != 0]])          # every distance is achieved
    assert got[got != INF].max() < 0xFFFFFFFE


def test_sssp_unit_weights_equal_bfs():
    g = gg.rmat(10, 8)
    g1 = gg.Graph(g.V, g.offsets, g.src, np.ones(g.E, dtype=np.uint32))
    np.testing.assert_array_equal(oracle.sssp_dijkstra(g1, 0), oracle.bfs_push(g, 0))
    np.testing.assert_array_equal(oracle.sssp_pull(g1, 0), oracle.bfs_push(g, 0))


def test_grid_weights_symmetric():
    g = gg.grid(12, 0.1).with_weights(1000)
    dst = g.dst()
    lookup = {(int(u), int(v)): int(w) for u, v, w in zip(g.src, dst, g.w)}
    for (u, v), w in lookup.items():
        assert lookup[(v, u)] == w
        assert 1 <= w <= 1000
