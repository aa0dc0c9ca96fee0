"""Pins for the oracle's Wedge Frontier, fullness and Wedge runs: the
paper's worked example (Sections 3.1, 3.3, 3.4), agreement of the
definition with the paper's edge-index transformation (Section 4), and the
invariants the paper states (Sections 3.2, 3.4, 5)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _golden import edges, read

EX = read("paper_example_fig4.txt")


def _example():
    s, d = edges(EX["edges"])
    return gg.from_edges(int(EX["V"][0]), s, d)


def test_paper_example_counts():
    g = _example()
    front = [int(x) for x in EX["frontier"]]
    dst = g.dst()
    active = np.isin(g.src, front)
    assert int(active.sum()) == int(EX["active_edges"][0])
    assert sorted(set(dst[active].tolist())) == [int(x) for x in EX["active_destinations"]]
    # a destination-oriented vertex frontier pulls every in-edge of those vertices
    dest_front = np.isin(dst, [int(x) for x in EX["active_destinations"]])
    assert int(dest_front.sum()) == int(EX["destination_frontier_edges"][0])
    assert oracle.fullness(g, front) == int(EX["fullness"][0])


def test_paper_example_wedge_frontier():
    g = _example()
    front = [int(x) for x in EX["frontier"]]
    for group, key in ((1, "wedge_group1"), (2, "wedge_group2")):
        want = [int(x) for x in EX[key]]
        assert oracle.wedge_groups_scan(g, front, group).tolist() == want
        assert oracle.wedge_groups_index(g, front, group).tolist() == want
    # two edges per group: every group adds at most one superfluous edge
    groups = oracle.wedge_groups_scan(g, front, 2)
    covered = np.concatenate([np.arange(2 * int(q), min(2 * int(q) + 2, g.E)) for q in groups])
    superfluous = (~np.isin(g.src[covered], front)).sum()
    assert superfluous <= len(groups) * (2 - 1)


def _random_frontier(V, frac, seed):
    r = np.array([gg.rand(seed, i) for i in range(V)], dtype=np.uint64)
    return (r % np.uint64(1000)) < np.uint64(int(frac * 1000))


@pytest.mark.parametrize("group", [1, 32, 64, 128, 512])
def test_transform_definition_equals_edge_index_walk(group):
    g = gg.rmat(12, 16)
    idx = oracle.edge_index(g, group)
    for frac, seed in ((0.001, 1), (0.02, 2), (0.3, 3)):
        f = _random_frontier(g.V, frac, seed)
        a = oracle.wedge_groups_scan(g, f, group)
        b = oracle.wedge_groups_index(g, f, group, index=idx)
        np.testing.assert_array_equal(a, b)
        # cover: every active edge lies in a listed group
        act = np.flatnonzero(f[g.src])
        assert np.all(np.isin(act // group, a))
        # exact: every listed group holds an active edge
        assert np.all(np.isin(a, act // group))
        assert oracle.fullness(g, f) == act.size


def test_coarsening_is_a_shift_and_union_is_preserved():
    g = gg.rmat(11, 16)
    f1 = _random_frontier(g.V, 0.01, 7)
    f2 = _random_frontier(g.V, 0.01, 8)
    fine = oracle.wedge_groups_scan(g, f1, 32)
    for k in range(1, 5):
        coarse = oracle.wedge_groups_scan(g, f1, 32 << k)
        np.testing.assert_array_equal(coarse, np.unique(fine >> k))
    both = oracle.wedge_groups_scan(g, f1 | f2, 32)
    np.testing.assert_array_equal(both, np.union1d(fine, oracle.wedge_groups_scan(g, f2, 32)))


def test_edge_index_rows_are_sorted_unique_and_complete():
    g = gg.rmat(10, 8)
    eo, ei = oracle.edge_index(g, 32)
    for u in range(0, g.V, 37):
        row = ei[eo[u]:eo[u + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0)
        want = np.unique(np.flatnonzero(g.src == u) // 32)
        np.testing.assert_array_equal(row, want)


@pytest.mark.parametrize("app", ["bfs", "cc", "sssp"])
def test_wedge_runs_reach_the_plain_result(app):
    """The Wedge Frontier carries the same information as the vertex frontier
    (Section 3.3) and coarser groups never break correctness (Section 3.4):
    every policy and precision reaches the definition's result."""
    base = gg.rmat(11, 16)
    if app == "cc":
        g = gg.symmetrize(base)
        want = oracle.cc_union_find(g)
    elif app == "sssp":
        g = base.with_weights(255)
        want = oracle.sssp_dijkstra(g, 0)
    else:
        g = base
        want = oracle.bfs_push(g, 0)
    for policy, tau, group in ((oracle.POLICY_ALWAYS_DENSE, 0, 32),
                               (oracle.POLICY_ALWAYS_SPARSE, 0, 32),
                               (oracle.POLICY_ALWAYS_SPARSE, 0, 1),
                               (oracle.POLICY_THRESHOLD, 100, 256),
                               (oracle.POLICY_THRESHOLD, 2000, 128)):
        vals, trace = oracle.wedge_run(app, g, 0, policy, tau, group)
        np.testing.assert_array_equal(vals, want)
        if policy == oracle.POLICY_ALWAYS_DENSE:
            assert trace[:, 2].sum() == 0
        if policy == oracle.POLICY_ALWAYS_SPARSE:
            assert trace[:, 2].min() == 1


def test_bfs_trace_follows_levels():
    """In BFS each vertex is in the frontier for exactly one iteration
    (Section 5): F_t is the level-t set, so |F_t| and fullness(F_t) follow
    from the levels alone; the fullness decision uses the strict test."""
    g = gg.rmat(12, 16)
    lvl = oracle.bfs_push(g, 0)
    od = oracle.outdeg(g)
    tau = 100
    _, trace = oracle.wedge_run("bfs", g, 0, oracle.POLICY_THRESHOLD, tau, 64)
    depth = int(lvl[lvl != oracle.INF].max())
    assert trace.shape[0] == depth + 1
    for t in range(depth + 1):
        members = lvl == t
        assert trace[t, 0] == members.sum()
        assert trace[t, 1] == od[members].sum()
        assert trace[t, 2] == int(trace[t, 1] * 10000 < tau * g.E)
        if trace[t, 2]:
            assert trace[t, 3] == oracle.wedge_groups_scan(g, members, 64).size


def _jacobi_frontiers(app, g, root):
    """Synchronous iteration written with NumPy, independently of the oracle:
    x_{t+1}[v] = min(x_t[v], min over in-edges (u, v) with u in F_t of
    x_t[u] (+ w)), F_{t+1} = {v : x_{t+1}[v] < x_t[v]}; returns the frontiers.
    Sources outside F_t offer nothing new (their value was offered before)."""
    V = g.V
    dst = g.dst().astype(np.int64)
    src = g.src.astype(np.int64)
    inf = np.iinfo(np.int64).max
    if app == "cc":
        x = np.arange(V, dtype=np.int64)
        front = np.ones(V, dtype=bool)
    else:
        x = np.full(V, inf, dtype=np.int64)
        x[root] = 0
        front = np.zeros(V, dtype=bool)
        front[root] = True
    w = g.w.astype(np.int64) if app == "sssp" else np.zeros(src.size, dtype=np.int64)
    fronts = []
    while front.any():
        fronts.append(front.copy())
        act = front[src]
        cand = np.full(V, inf, dtype=np.int64)
        vals = np.minimum(x[src[act]] + w[act], 0xFFFFFFFE) if app == "sssp" else x[src[act]]
        np.minimum.at(cand, dst[act], vals)
        nx = np.minimum(x, cand)
        front = nx < x
        x = nx
    return fronts


@pytest.mark.parametrize("app", ["cc", "sssp"])
def test_synchronous_cc_sssp_traces_follow_jacobi(app):
    """The oracle's Wedge run is synchronous for CC and SSSP: its frontier
    sizes, fullness and decisions per iteration equal those of the plain
    Jacobi iteration (the reference the GPU's synchronous mode is held to)."""
    base = gg.rmat(11, 16)
    g = gg.symmetrize(base) if app == "cc" else base.with_weights(255)
    od = oracle.outdeg(g)
    tau = 2000
    fronts = _jacobi_frontiers(app, g, 0)
    _, trace = oracle.wedge_run(app, g, 0, oracle.POLICY_THRESHOLD, tau, 32)
    assert trace.shape[0] == len(fronts)
    for t, f in enumerate(fronts):
        assert trace[t, 0] == f.sum()
        assert trace[t, 1] == od[f].sum()
        assert trace[t, 2] == int(trace[t, 1] * 10000 < tau * g.E)
        if trace[t, 2]:
            assert trace[t, 3] == oracle.wedge_groups_scan(g, f, 32).size
