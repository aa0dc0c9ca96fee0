"""The oracle's pins have teeth: the checks they rest on (SciPy's graph
routines, the invariants of the definitions, PageRank's mass and closed
forms) accept the oracle's results and reject plausible mistakes planted
on the CPU -- an off-by-one level, a dropped or reversed edge, a shifted
weight, max instead of min, a lost dangling mass, a teleport term not
divided by V, a contribution not divided by the out-degree."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import graphgen as gg
import oracle

INF = oracle.INF


def _adj(g, w=None):
    data = np.ones(g.E) if w is None else w.astype(np.float64)
    return sp.csr_matrix((data, (g.src.astype(np.int64), g.dst().astype(np.int64))), shape=(g.V, g.V))


def _u32(d):
    return np.where(np.isinf(d), INF, d).astype(np.uint32)


def bfs_ok(g, root, lvl):
    want = _u32(csg.shortest_path(_adj(g), directed=True, unweighted=True, indices=root))
    if not np.array_equal(lvl, want):
        return False
    src, dst = g.src.astype(np.int64), g.dst().astype(np.int64)
    lu, lv = lvl[src].astype(np.int64), lvl[dst].astype(np.int64)
    fin = lu != INF
    if lvl[root] != 0 or np.any(lv[fin] > lu[fin] + 1):
        return False
    parent = np.zeros(g.V, dtype=bool)
    parent[dst[fin & (lv == lu + 1)]] = True
    reached = np.flatnonzero(lvl != INF)
    return bool(np.all(parent[reached[reached != root]]))


def sssp_ok(g, root, d):
    want = _u32(csg.dijkstra(_adj(g, g.w), directed=True, indices=root))
    return bool(np.array_equal(d, want))


def cc_ok(g, labels):
    _, comp = csg.connected_components(_adj(g), directed=False)
    want = np.empty(g.V, dtype=np.int64)
    mins = np.full(comp.max() + 1, np.iinfo(np.int64).max)
    np.minimum.at(mins, comp, np.arange(g.V))
    want[:] = mins[comp]
    return bool(np.array_equal(labels.astype(np.int64), want))


def pr_ok(g, pr):
    """Mass 1, every rank at least the teleport share, and the rank of a
    directed cycle uniform (checked separately)."""
    return abs(pr.sum() - 1.0) < 1e-12 and bool(np.all(pr >= 0.15 / g.V * (1 - 1e-12)))


def _pr_numpy(g, d=0.85, iters=20, dangling=True, teleport_over_v=True, divide=True):
    """PageRank restated with NumPy, with optional planted mistakes."""
    V = g.V
    od = np.bincount(g.src.astype(np.int64), minlength=V).astype(np.float64)
    dst = g.dst().astype(np.int64)
    src = g.src.astype(np.int64)
    pr = np.full(V, 1.0 / V)
    for _ in range(iters):
        contrib = np.where(od > 0, pr / np.maximum(od, 1), 0.0) if divide else np.where(od > 0, pr, 0.0)
        s = np.zeros(V)
        np.add.at(s, dst, contrib[src])
        D = pr[od == 0].sum() if dangling else 0.0
        base = (1 - d) / V if teleport_over_v else (1 - d)
        pr = base + d * (s + D / V)
    return pr


def test_bfs_pins_reject_planted_mistakes():
    g = gg.rmat(10, 8)
    lvl = oracle.bfs_push(g, 0)
    assert bfs_ok(g, 0, lvl)
    off_by_one = np.where((lvl != INF) & (np.arange(g.V) != 0), lvl + 1, lvl).astype(np.uint32)
    assert not bfs_ok(g, 0, off_by_one)
    # the edges reversed (pushing along in-edges)
    rev = gg.from_edges(g.V, g.dst(), g.src)
    assert not bfs_ok(g, 0, oracle.bfs_push(rev, 0))
    # one edge of the root dropped
    keep = np.ones(g.E, dtype=bool)
    keep[np.flatnonzero(g.src == 0)[0]] = False
    dropped = gg.from_edges(g.V, g.src[keep], g.dst()[keep])
    assert not bfs_ok(g, 0, oracle.bfs_push(dropped, 0))


def test_sssp_pins_reject_planted_mistakes():
    g = gg.rmat(10, 8).with_weights(255)
    d = oracle.sssp_dijkstra(g, 0)
    assert sssp_ok(g, 0, d)
    shifted = gg.Graph(g.V, g.offsets, g.src, g.w + 1)
    assert not sssp_ok(g, 0, oracle.sssp_dijkstra(shifted, 0))
    unit = gg.Graph(g.V, g.offsets, g.src, np.ones(g.E, dtype=np.uint32))
    assert not sssp_ok(g, 0, oracle.sssp_dijkstra(unit, 0))


def test_cc_pins_reject_planted_mistakes():
    g = gg.symmetrize(gg.rmat(10, 2))
    labels = oracle.cc_union_find(g)
    assert cc_ok(g, labels)
    _, comp = csg.connected_components(_adj(g), directed=False)
    maxs = np.zeros(comp.max() + 1, dtype=np.int64)
    np.maximum.at(maxs, comp, np.arange(g.V))
    assert not cc_ok(g, maxs[comp])
    # label propagation pulled over the unsymmetrised in-edges only
    directed = gg.rmat(10, 2)
    assert cc_ok(gg.symmetrize(directed), oracle.cc_pull(gg.symmetrize(directed)))
    assert not cc_ok(gg.symmetrize(directed), oracle.cc_pull(directed))


def test_pagerank_pins_reject_planted_mistakes():
    g = gg.rmat(9, 6)  # has vertices of out-degree 0
    assert np.any(np.bincount(g.src.astype(np.int64), minlength=g.V) == 0)
    assert pr_ok(g, oracle.pr_pull(g, 0.85, 20))
    np.testing.assert_allclose(_pr_numpy(g), oracle.pr_pull(g, 0.85, 20), rtol=1e-12)
    assert not pr_ok(g, _pr_numpy(g, dangling=False))
    assert not pr_ok(g, _pr_numpy(g, teleport_over_v=False))
    assert not pr_ok(g, _pr_numpy(g, divide=False))


def test_wedge_frontier_fixture_rejects_planted_mistakes():
    """The worked example's Wedge Frontiers (one and two edges per group)
    single out the definition: groups of the active sources' out-edges.
    Destination-oriented groups, an off-by-one group index or the sources'
    in-edges all miss them."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from _golden import edges, read
    ex = read("paper_example_fig4.txt")
    s, d = edges(ex["edges"])
    g = gg.from_edges(int(ex["V"][0]), s, d)
    front = [int(x) for x in ex["frontier"]]
    src, dst = g.src.astype(np.int64), g.dst().astype(np.int64)
    pos = np.arange(g.E)

    def groups(active, size, shift=0):
        return sorted(set(((pos[active] + shift) // size).tolist()))

    for size, key in ((1, "wedge_group1"), (2, "wedge_group2")):
        want = [int(x) for x in ex[key]]
        assert groups(np.isin(src, front), size) == want                   # the definition
        assert groups(np.isin(dst, front), size) != want                   # destination-oriented
        assert groups(np.isin(src, front), size, shift=1) != want          # off by one position
        assert oracle.wedge_groups_scan(g, front, size).tolist() == want
    active_dst = sorted(set(dst[np.isin(src, front)].tolist()))
    assert active_dst == [int(x) for x in ex["active_destinations"]]
    # in-edges of the frontier instead of its out-edges
    assert sorted(set(src[np.isin(dst, front)].tolist())) != active_dst
