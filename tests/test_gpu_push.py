"""The push/pull hybrid (the comparison engine: sparse iterations push over
the frontier's out-edges, dense ones pull), through the C ABI, against the
oracle: levels, labels and distances bit for bit under every policy, and
BFS's level-synchronous trace (frontier size, fullness, decision) iteration
by iteration."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _gpu import empty_u32, graph, opts, u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu

POLICIES = {"threshold": None, "push": wedge.SWITCH_ALWAYS_SPARSE, "pull": wedge.SWITCH_ALWAYS_DENSE}


def _push_opts(app, policy, tau=None, trace=0):
    o = opts(app, switch=POLICIES[policy], tau=tau, trace=trace)
    o.sparse_push = 1
    return o


def _run(G, app, root, o):
    out = empty_u32(G.V)
    f = {"bfs": lambda: wedge.wedge_run_bfs(G.handle, root, out, o),
         "cc": lambda: wedge.wedge_run_cc(G.handle, out, o),
         "sssp": lambda: wedge.wedge_run_sssp(G.handle, root, out, o)}[app]
    st = f()
    return u32(out)[: G.V], st


@pytest.fixture(scope="module")
def rmat():
    return gg.rmat(16, 16).with_weights(255)


@pytest.fixture(scope="module")
def rmat_dev(rmat):
    G = graph(rmat)
    yield G
    G.close()


@pytest.fixture(scope="module")
def sym():
    return gg.symmetrize(gg.rmat(15, 8))


@pytest.fixture(scope="module")
def sym_dev(sym):
    G = graph(sym, with_weights=False)
    yield G
    G.close()


@pytest.mark.parametrize("policy,tau", [("threshold", None), ("threshold", 2000), ("push", None), ("pull", None)])
@pytest.mark.parametrize("trace", [0, 1])
def test_hybrid_matches_oracle(rmat, rmat_dev, sym, sym_dev, policy, tau, trace):
    for root in (0, 777):
        got, st = _run(rmat_dev, "bfs", root, _push_opts("bfs", policy, tau, trace))
        np.testing.assert_array_equal(got, oracle.bfs_push(rmat, root))
        if policy == "push":
            assert st.sparse_iters == st.iters
        got, _ = _run(rmat_dev, "sssp", root, _push_opts("sssp", policy, tau, trace))
        np.testing.assert_array_equal(got, oracle.sssp_dijkstra(rmat, root))
    got, _ = _run(sym_dev, "cc", 0, _push_opts("cc", policy, tau, trace))
    np.testing.assert_array_equal(got, oracle.cc_union_find(sym))


@pytest.mark.parametrize("tau", [100, 2000, 10000])
def test_hybrid_bfs_trace_matches_oracle(rmat, rmat_dev, tau):
    """BFS is level-synchronous in both engines, so the hybrid takes the
    oracle's decisions; a push iteration pushes exactly the frontier's
    out-edges (the fullness)."""
    got, st = _run(rmat_dev, "bfs", 0, _push_opts("bfs", "threshold", tau, trace=1))
    tr = wedge.wedge_get_trace(rmat_dev.handle)
    _, ot = oracle.wedge_run("bfs", rmat, 0, oracle.POLICY_THRESHOLD, tau, 32)
    assert len(tr) == ot.shape[0] == st.iters
    for t, rec in enumerate(tr):
        assert rec["nfront"] == ot[t, 0], t
        assert rec["fullness"] == ot[t, 1], t
        assert rec["mode"] == ot[t, 2], t
    pushed = sum(int(ot[t, 1]) for t in range(len(tr)) if ot[t, 2])
    dense = sum(1 for t in range(len(tr)) if not ot[t, 2])
    assert st.edges_pulled == pushed + dense * rmat.src.size


def _small_cases():
    cases = [gg.random_graph(V, m, seed=950 + i) for i, (V, m) in
             enumerate([(1, 0), (7, 0), (5, 3), (40, 37), (300, 1201), (4096, 70001)])]
    cases.append(gg.grid(48, 0.02))
    V = 50_000
    v = np.arange(V, dtype=np.int64)
    cases.append(gg.from_edges(V, np.concatenate([(v * 7919 + 1) % V, ((v * 31 + 5) % V)[v % 3 == 0]]),
                               np.concatenate([v, v[v % 3 == 0]])))
    return cases


@pytest.mark.parametrize("idx", range(8))
@pytest.mark.parametrize("policy", ["threshold", "push"])
def test_hybrid_small_and_degenerate_graphs(idx, policy):
    g = _small_cases()[idx].with_weights(1000)
    G = graph(g)
    try:
        for root in sorted({0, g.V - 1, g.V // 2}):
            got, _ = _run(G, "bfs", root, _push_opts("bfs", policy))
            np.testing.assert_array_equal(got, oracle.bfs_push(g, root))
            got, _ = _run(G, "sssp", root, _push_opts("sssp", policy))
            np.testing.assert_array_equal(got, oracle.sssp_dijkstra(g, root))
    finally:
        G.close()
    s = gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))
    S = graph(s, with_weights=False)
    try:
        got, _ = _run(S, "cc", 0, _push_opts("cc", policy))
        np.testing.assert_array_equal(got, oracle.cc_union_find(s))
    finally:
        S.close()


def test_hybrid_and_wedge_share_a_graph(rmat, rmat_dev):
    """Runs of both engines on one graph object, interleaved, stay exact."""
    want = oracle.sssp_dijkstra(rmat, 5)
    for push in (1, 0, 1):
        o = opts("sssp")
        o.sparse_push = push
        got, _ = _run(rmat_dev, "sssp", 5, o)
        np.testing.assert_array_equal(got, want)


def test_push_with_synchronous_is_rejected(rmat_dev):
    o = opts("sssp")
    o.sparse_push = 1
    o.synchronous = 1
    with pytest.raises(wedge.WedgeError):
        _run(rmat_dev, "sssp", 0, o)
