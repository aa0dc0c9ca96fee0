"""The paper's finer Wedge Frontier precisions (Section 3.4, "Frontier
Precision"; the tuned CC/SSSP setting of Section 5.2 is 4 edge vectors, up
to 16 edges, per bit): log2_coarsen = -1 / -2 (as uint32) gives entries of
16 / 8 edges.  The transformation must equal the definition at those group
sizes, runs must reach the oracle's results under every policy, and the
synchronous traces (frontier, fullness, decision, entries per iteration)
must equal the oracle's Wedge run with the same group size."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _gpu import bitmap, dev_u32, empty_u32, graph, opts, u32, zeros_u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu

FINE = {-1: 16, -2: 8}


def _u(k):
    return k & 0xFFFFFFFF


@pytest.fixture(scope="module")
def g16():
    return gg.rmat(16, 16).with_weights(255)


@pytest.fixture(scope="module")
def G16(g16):
    G = graph(g16)
    yield G
    G.close()


@pytest.fixture(scope="module")
def s15():
    g = gg.rmat(15, 16, seed=3)
    return gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))


@pytest.fixture(scope="module")
def S15(s15):
    S = graph(s15, with_weights=False)
    yield S
    S.close()


def _run(G, app, o, root=0):
    out = empty_u32(G.V)
    if app == "bfs":
        st = wedge.wedge_run_bfs(G.handle, root, out, o)
    elif app == "cc":
        st = wedge.wedge_run_cc(G.handle, out, o)
    else:
        st = wedge.wedge_run_sssp(G.handle, root, out, o)
    return u32(out)[: G.V], st


@pytest.mark.parametrize("k", [-1, -2])
@pytest.mark.parametrize("frac", [0.0002, 0.01, 0.2, 1.0])
def test_transform_matches_definition(g16, G16, k, frac):
    r = np.array([gg.rand(83, i) for i in range(g16.V)], dtype=np.uint64)
    front = (r % np.uint64(100000)) < np.uint64(int(frac * 100000))
    front[0] = True  # the hub: a long row
    cap = (g16.E + FINE[k] - 1) // FINE[k]
    lst = empty_u32(cap)
    cnt = zeros_u32(1)
    wedge.wedge_frontier_transform(G16.handle, dev_u32(bitmap(g16.V, front)), _u(k), lst, cnt)
    n = int(u32(cnt)[0])
    got = u32(lst)[:n].astype(np.uint64)
    assert np.unique(got).size == n
    np.testing.assert_array_equal(np.sort(got), oracle.wedge_groups_scan(g16, front, FINE[k]))


@pytest.mark.parametrize("k", [-1, -2])
@pytest.mark.parametrize("policy", ["threshold", "sparse", "tau50"])
def test_runs_match_oracle(g16, G16, s15, S15, k, policy):
    sw = {"threshold": None, "sparse": wedge.SWITCH_ALWAYS_SPARSE, "tau50": None}[policy]
    tau = {"threshold": None, "sparse": None, "tau50": 5000}[policy]
    got, st = _run(G16, "bfs", opts("bfs", switch=sw, tau=tau, k=_u(k)))
    np.testing.assert_array_equal(got, oracle.bfs_push(g16, 0))
    got, _ = _run(G16, "sssp", opts("sssp", switch=sw, tau=tau, k=_u(k)))
    np.testing.assert_array_equal(got, oracle.sssp_dijkstra(g16, 0))
    got, _ = _run(S15, "cc", opts("cc", switch=sw, tau=tau, k=_u(k)))
    np.testing.assert_array_equal(got, oracle.cc_union_find(s15))
    if policy == "sparse":
        assert st.sparse_iters == st.iters


@pytest.mark.parametrize("k", [-1, -2])
def test_bfs_trace_matches_oracle(g16, G16, k):
    o = opts("bfs", tau=2000, k=_u(k), trace=1)
    got, st = _run(G16, "bfs", o)
    tr = wedge.wedge_get_trace(G16.handle)
    _, ot = oracle.wedge_run("bfs", g16, 0, oracle.POLICY_THRESHOLD, 2000, FINE[k])
    assert len(tr) == ot.shape[0] == st.iters
    for t, rec in enumerate(tr):
        assert (rec["nfront"], rec["fullness"], rec["mode"]) == tuple(ot[t, :3]), t
        if rec["mode"]:
            assert rec["nchunks"] == ot[t, 3], t
            assert rec["log2_coarsen"] == _u(k)


@pytest.mark.parametrize("app", ["cc", "sssp"])
@pytest.mark.parametrize("k", [-1, -2])
def test_synchronous_trace_matches_oracle(g16, G16, s15, S15, app, k):
    g, G = (s15, S15) if app == "cc" else (g16, G16)
    o = opts(app, tau=2000, k=_u(k), trace=1)
    o.synchronous = 1
    got, st = _run(G, app, o)
    tr = wedge.wedge_get_trace(G.handle)
    want, ot = oracle.wedge_run(app, g, 0, oracle.POLICY_THRESHOLD, 2000, FINE[k])
    np.testing.assert_array_equal(got, want)
    assert len(tr) == ot.shape[0] == st.iters
    for t, rec in enumerate(tr):
        assert (rec["nfront"], rec["fullness"], rec["mode"]) == tuple(ot[t, :3]), t
        if rec["mode"]:
            assert rec["nchunks"] == ot[t, 3], t


def test_pull_iterate_over_a_fine_list(g16, G16):
    """One BFS pull over 8-edge entries listed by hand: exactly the
    destinations of the listed units' edges that leave the frontier (and
    were unreached) get level 1 (BFS pulls are level-synchronous, so the
    result does not depend on the schedule)."""
    import torch
    k = -2
    front = np.zeros(g16.V, dtype=bool)
    front[[0, 5, 77, 4000]] = True
    ents = oracle.wedge_groups_scan(g16, front, 8).astype(np.uint32)
    lvl = np.full(g16.V, 0xFFFFFFFF, dtype=np.uint32)
    lvl[front] = 0
    vals = dev_u32(lvl)
    nxt = zeros_u32((g16.V + 31) // 32)
    full = torch.zeros(1, dtype=torch.int64, device="cuda")
    nf = zeros_u32(1)
    wedge.wedge_pull_iterate(G16.handle, "bfs", vals, 0, dev_u32(bitmap(g16.V, front)), dev_u32(ents),
                             dev_u32([ents.size]), _u(k), nxt, full, nf)
    off = g16.offsets.astype(np.int64)
    dst = np.repeat(np.arange(g16.V), np.diff(off))
    pos = (ents[:, None].astype(np.int64) * 8 + np.arange(8)[None, :]).reshape(-1)
    pos = pos[pos < g16.E]
    hit = pos[front[g16.src[pos]]]
    want = lvl.copy()
    reached = np.unique(dst[hit])
    reached = reached[lvl[reached] == 0xFFFFFFFF]
    want[reached] = 1
    np.testing.assert_array_equal(u32(vals)[: g16.V], want)
    assert int(u32(nf)[0]) == reached.size
    od = oracle.outdeg(g16)
    assert int(full.item()) == int(od[reached].sum())


@pytest.mark.parametrize("case", ["empty", "one_vertex", "ragged"])
def test_degenerate_graphs(case):
    if case == "empty":
        g = gg.Graph(5, np.zeros(6, dtype=np.uint32), np.zeros(0, dtype=np.uint32)).with_weights(9)
    elif case == "one_vertex":
        g = gg.Graph(1, np.array([0, 1], dtype=np.uint32), np.array([0], dtype=np.uint32)).with_weights(9)
    else:
        g = gg.rmat(9, 7, seed=3).with_weights(40)
    G = graph(g)
    try:
        for k in (-1, -2):
            got, _ = _run(G, "bfs", opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=_u(k)))
            np.testing.assert_array_equal(got, oracle.bfs_push(g, 0))
            got, _ = _run(G, "sssp", opts("sssp", k=_u(k)))
            np.testing.assert_array_equal(got, oracle.sssp_dijkstra(g, 0))
    finally:
        G.close()


def test_invalid_precisions(G16):
    out = empty_u32(G16.V)
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_run_bfs(G16.handle, 0, out, opts("bfs", k=_u(-3)))
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_run_bfs(G16.handle, 0, out, opts("bfs", k=8))
    # batched runs list whole chunks: -1 acts as 0
    lv = empty_u32(G16.V * 4)
    roots = np.array([0, 9, 300, 4000], dtype=np.uint32)
    wedge.wedge_run_bfs_batch(G16.handle, roots, None, 4, lv, opts("bfs", k=_u(-1)))
    a = u32(lv)[: G16.V * 4].copy()
    wedge.wedge_run_bfs_batch(G16.handle, roots, None, 4, lv, opts("bfs", k=0))
    np.testing.assert_array_equal(u32(lv)[: G16.V * 4], a)
