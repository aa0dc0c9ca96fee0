"""Pins for the oracle's FP64 PageRank: hand-derived iterates, closed forms,
mass conservation and NetworkX's PageRank at the fixed point."""
import networkx as nx
import numpy as np
import pytest

import graphgen as gg
import oracle
from _golden import edges, read

G = read("pagerank_small.txt")


def _graph(key, V):
    s, d = edges(G[key + " edges"])
    return gg.from_edges(V, s, d)


def test_two_vertex_hand_derived():
    g = _graph("two_vertex", 2)
    for it, key in ((1, "iter1"), (2, "iter2")):
        want = np.array([float(x) for x in G["two_vertex " + key]])
        np.testing.assert_allclose(oracle.pr_pull(g, 0.85, it), want, rtol=0, atol=1e-15)
        np.testing.assert_allclose(oracle.pr_push(g, 0.85, it), want, rtol=0, atol=1e-15)
    fixed = np.array([float(x) for x in G["two_vertex fixed"]])
    np.testing.assert_allclose(oracle.pr_pull(g, 0.85, 300), fixed, rtol=0, atol=1e-14)


def test_star_hand_derived():
    g = _graph("star4", 4)
    want = np.array([float(x) for x in G["star4 iter1"]])
    np.testing.assert_allclose(oracle.pr_pull(g, 0.85, 1), want, rtol=0, atol=1e-15)


def test_cycle_and_empty_graph_stay_uniform():
    V = 37
    cyc = gg.from_edges(V, np.arange(V), (np.arange(V) + 1) % V)
    np.testing.assert_allclose(oracle.pr_pull(cyc, 0.85, 20), np.full(V, 1 / V), rtol=1e-13)
    empty = gg.from_edges(V, [], [])
    np.testing.assert_allclose(oracle.pr_pull(empty, 0.85, 20), np.full(V, 1 / V), rtol=1e-13)


@pytest.mark.parametrize("scale", [8, 11])
def test_mass_and_push_pull_agree(scale):
    g = gg.rmat(scale, 8)
    pull = oracle.pr_pull(g, 0.85, 20)
    push = oracle.pr_push(g, 0.85, 20)
    assert abs(pull.sum() - 1.0) < 1e-12
    np.testing.assert_allclose(pull, push, rtol=1e-12, atol=0)
    assert np.all(pull >= 0.15 / g.V * (1 - 1e-12))


def test_fixed_point_matches_networkx():
    g = gg.rmat(9, 6)  # has dangling vertices
    G_ = nx.DiGraph()
    G_.add_nodes_from(range(g.V))
    G_.add_edges_from(zip(g.src.tolist(), g.dst().tolist()))
    ref = nx.pagerank(G_, alpha=0.85, tol=1e-15, max_iter=2000)
    want = np.array([ref[v] for v in range(g.V)])
    got = oracle.pr_pull(g, 0.85, 400)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_in_sums_hand_graph_and_identities():
    # 0->2, 1->2, 3->2, 2->0: in-sums by hand
    g = gg.from_edges(4, [0, 1, 3, 2], [2, 2, 2, 0])
    x = np.array([1.0, 10.0, 100.0, 1000.0])
    np.testing.assert_array_equal(oracle.in_sums(g, x), [100.0, 0.0, 1011.0, 0.0])
    # every source value is counted once per out-edge
    h = gg.rmat(10, 8, seed=5)
    y = np.random.default_rng(1).random(h.V)
    od = oracle.outdeg(h).astype(np.float64)
    assert abs(oracle.in_sums(h, y).sum() - (y * od).sum()) < 1e-9 * (y * od).sum()


def test_in_sums_is_pagerank_first_pass():
    # with d = 1, one PageRank iterate is the in-edge sum of pr0/outdeg plus D/V
    g = gg.rmat(10, 8, seed=6)
    V = g.V
    od = oracle.outdeg(g)
    pr0 = np.full(V, 1.0 / V)
    contrib = np.where(od > 0, pr0 / np.maximum(od, 1), 0.0)
    D = pr0[od == 0].sum()
    np.testing.assert_allclose(oracle.in_sums(g, contrib) + D / V, oracle.pr_pull(g, 1.0, 1), rtol=1e-13, atol=0)
