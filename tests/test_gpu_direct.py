"""A run's transformation expands the listed rows directly (in the scan
kernel, without work pieces) when the frontier list is complete and every
row has at most 32 edge-index entries; otherwise it cuts pieces.  Both paths
must give the oracle's results and the Wedge Frontier sizes of the oracle's
run; the traces show which path served each sparse iteration (npieces = 0
with a non-empty Wedge Frontier: the direct path)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _gpu import empty_u32, graph, opts, u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu


def _trace_run(G, app, root, o):
    out = empty_u32(G.V)
    if app == "bfs":
        wedge.wedge_run_bfs(G.handle, root, out, o)
    else:
        wedge.wedge_run_sssp(G.handle, root, out, o)
    return u32(out)[: G.V].copy(), wedge.wedge_get_trace(G.handle)


@pytest.mark.parametrize("app", ["bfs", "sssp"])
def test_grid_rows_go_direct(app):
    g = gg.grid(96, 0.02).with_weights(50)  # rows of at most 4 chunks
    G = graph(g)
    try:
        want = oracle.bfs_push(g, 5) if app == "bfs" else oracle.sssp_dijkstra(g, 5)
        for k in (0, 2):
            got, tr = _trace_run(G, app, 5, opts(app, switch=wedge.SWITCH_ALWAYS_SPARSE, k=k, trace=1))
            np.testing.assert_array_equal(got, want)
            sparse = [r for r in tr if r["mode"] == 1 and r["nchunks"] > 0]
            assert sparse and all(r["npieces"] == 0 for r in sparse)
            # the device loop (no trace) takes the same path
            out = empty_u32(G.V)
            o = opts(app, switch=wedge.SWITCH_ALWAYS_SPARSE, k=k)
            (wedge.wedge_run_bfs if app == "bfs" else wedge.wedge_run_sssp)(G.handle, 5, out, o, False)
            np.testing.assert_array_equal(u32(out)[: G.V], want)
    finally:
        G.close()


def test_rmat_mixes_direct_and_pieces():
    g = gg.rmat(15, 16).with_weights(255)
    G = graph(g)
    try:
        seen = set()
        for root in (0, 77, 3001, 12345):
            for app in ("bfs", "sssp"):
                o = opts(app, tau=2000, k=0, trace=1)
                got, tr = _trace_run(G, app, root, o)
                want = oracle.bfs_push(g, root) if app == "bfs" else oracle.sssp_dijkstra(g, root)
                np.testing.assert_array_equal(got, want)
                if app == "bfs":  # level-synchronous: the oracle's run has the same Wedge Frontiers
                    _, ot = oracle.wedge_run("bfs", g, root, oracle.POLICY_THRESHOLD, 2000, 32)
                    assert [r["nchunks"] for r in tr if r["mode"]] == [int(x[3]) for x in ot if x[2]]
                for r in tr:
                    if r["mode"] == 1 and r["nchunks"] > 0:
                        seen.add("direct" if r["npieces"] == 0 else "pieces")
        assert seen == {"direct", "pieces"}
    finally:
        G.close()


def test_frontier_with_one_long_row_takes_pieces():
    # a star: the hub's row holds every chunk, so its frontier is cut into pieces
    V = 5000
    src = [0] * (V - 1) + list(range(1, V))
    dst = list(range(1, V)) + [0] * (V - 1)
    g = gg.from_edges(V, src, dst)
    G = graph(g, with_weights=False)
    try:
        got, tr = _trace_run(G, "bfs", 0, opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, trace=1))
        np.testing.assert_array_equal(got, oracle.bfs_push(g, 0))
        first = [r for r in tr if r["mode"] == 1 and r["nchunks"] > 0][0]
        assert first["npieces"] > 0
    finally:
        G.close()
