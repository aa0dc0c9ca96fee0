"""The compressed edge index (Section 4: in-memory compression of the edge
index to cut the transformation's memory traffic): with wedge_tuning's
edge_index = 1 the transformation decodes blocks of up to 32 sorted
entries (first entry + packed differences).  Its Wedge Frontier must equal
the definition and the oracle's walk of the edge index at every precision,
single rows of every length class must decode to exactly their entries,
and whole runs must reach the oracle's results."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _gpu import bitmap, dev_u32, empty_u32, graph, opts, u32, zeros_u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g16():
    return gg.rmat(16, 16).with_weights(255)


@pytest.fixture(scope="module")
def G16(g16):
    G = graph(g16)
    wedge.wedge_graph_set_tuning(G.handle, edge_index=1)
    yield G
    G.close()


def _transform(G, front, k):
    nc = G.info["nchunks"]
    lst = empty_u32((nc + (1 << k) - 1) >> k)
    cnt = zeros_u32(1)
    wedge.wedge_frontier_transform(G.handle, dev_u32(bitmap(G.V, front)), k, lst, cnt)
    n = int(u32(cnt)[0])
    got = u32(lst)[:n].astype(np.uint64)
    assert np.unique(got).size == n, "entries must be distinct"
    return np.sort(got)


def _decode(zbo, zhdr, zwords, eo):
    """Rows of the compressed index, decoded on the host from its documented
    layout (include/wedge.h, wedge_graph_copy_edge_index_z)."""
    rows = []
    for u in range(len(eo) - 1):
        n_row = int(eo[u + 1] - eo[u])
        out = []
        for b in range(int(zbo[u]), int(zbo[u + 1])):
            hx, hy = int(zhdr[2 * b]), int(zhdr[2 * b + 1])
            w, x = hx >> 27, hx & 0x7FFFFFF
            n = min(32, n_row - len(out))
            vals = [x]
            for i in range(1, n):
                bit = (i - 1) * w
                j, r = bit >> 5, bit & 31
                two = int(zwords[hy + j]) | ((int(zwords[hy + j + 1]) << 32) if hy + j + 1 < len(zwords) else 0)
                vals.append(vals[-1] + ((two >> r) & ((1 << w) - 1)))
            out += vals
        rows.append(out)
    return rows


def test_compressed_index_decodes_to_the_rows(g16, G16):
    info = wedge.wedge_graph_get_info(G16.handle)
    zbo = empty_u32(G16.V + 1)
    zhdr = empty_u32(2 * info["eidx_z_blocks"])
    zwords = empty_u32(info["eidx_z_words"])
    wedge.wedge_graph_copy_edge_index_z(G16.handle, zbo, zhdr, zwords)
    zbo, zhdr, zwords = u32(zbo)[: G16.V + 1], u32(zhdr), u32(zwords)[: info["eidx_z_words"]]
    eo, ei = oracle.edge_index(g16, 32)
    nb = (np.diff(eo.astype(np.int64)) + 31) // 32
    np.testing.assert_array_equal(zbo.astype(np.int64), np.concatenate([[0], np.cumsum(nb)]))
    rows = _decode(zbo, zhdr, zwords, eo)
    for u in range(G16.V):
        assert rows[u] == [int(x) for x in ei[eo[u]:eo[u + 1]]], u


def test_compressed_index_is_smaller(G16):
    info = wedge.wedge_graph_get_info(G16.handle)
    assert wedge.wedge_graph_get_tuning(G16.handle)["edge_index"] == 1
    assert 0 < info["eidx_z_bytes"] < info["eidx_bytes"]


@pytest.mark.parametrize("frac", [0.0005, 0.02, 0.3, 1.0])
def test_transform_matches_definition(g16, G16, frac):
    r = np.array([gg.rand(81, i) for i in range(g16.V)], dtype=np.uint64)
    front = (r % np.uint64(100000)) < np.uint64(int(frac * 100000))
    front[0] = True
    idx = oracle.edge_index(g16, 32)
    for k in (0, 1, 3, 7):
        got = _transform(G16, front, k)
        np.testing.assert_array_equal(got, oracle.wedge_groups_scan(g16, front, 32 << k))
        np.testing.assert_array_equal(got, np.unique(oracle.wedge_groups_index(g16, front, 32, idx) >> np.uint64(k)))


def test_single_rows_decode_exactly(g16, G16):
    """One-vertex frontiers: the hub, rows of 1, 31, 32, 33, 63, 64, 65 and
    97 entries (block boundaries and ragged tails) and the longest rows."""
    eo, ei = oracle.edge_index(g16, 32)
    lens = np.diff(eo.astype(np.int64))
    picks = {0, int(np.argmax(lens))}
    for L in (1, 31, 32, 33, 63, 64, 65, 97):
        c = np.flatnonzero(lens == L)
        if c.size:
            picks.add(int(c[0]))
    picks |= set(np.argsort(lens)[-5:].tolist())
    assert len(picks) >= 8
    for u in sorted(picks):
        front = np.zeros(g16.V, dtype=bool)
        front[u] = True
        want = ei[eo[u]:eo[u + 1]]
        np.testing.assert_array_equal(_transform(G16, front, 0), want)
        np.testing.assert_array_equal(_transform(G16, front, 2), np.unique(want >> np.uint64(2)))


@pytest.mark.parametrize("mode", ["default", "sparse0", "sparse2", "tau50k0"])
def test_runs_match_oracle(g16, G16, mode):
    extra = {"default": {}, "sparse0": {"switch": wedge.SWITCH_ALWAYS_SPARSE, "k": 0},
             "sparse2": {"switch": wedge.SWITCH_ALWAYS_SPARSE, "k": 2}, "tau50k0": {"tau": 5000, "k": 0}}[mode]
    out = empty_u32(g16.V)
    wedge.wedge_run_bfs(G16.handle, 0, out, opts("bfs", **extra))
    np.testing.assert_array_equal(u32(out)[: g16.V], oracle.bfs_push(g16, 0))
    wedge.wedge_run_sssp(G16.handle, 0, out, opts("sssp", **extra))
    np.testing.assert_array_equal(u32(out)[: g16.V], oracle.sssp_dijkstra(g16, 0))
    s = gg.symmetrize(gg.Graph(g16.V, g16.offsets, g16.src))
    S = graph(s, with_weights=False)
    try:
        wedge.wedge_graph_set_tuning(S.handle, edge_index=1)
        wedge.wedge_run_cc(S.handle, out, opts("cc", **extra))
        np.testing.assert_array_equal(u32(out)[: s.V], oracle.cc_union_find(s))
    finally:
        S.close()


@pytest.mark.parametrize("case", ["empty", "one_vertex", "ragged", "caller_index"])
def test_degenerate_graphs(case):
    """E = 0, V = 1, a graph whose last row and chunk are ragged, and a
    caller's edge index with duplicate entries (zero differences)."""
    if case == "empty":
        g = gg.Graph(5, np.zeros(6, dtype=np.uint32), np.zeros(0, dtype=np.uint32))
    elif case == "one_vertex":
        g = gg.Graph(1, np.array([0, 1], dtype=np.uint32), np.array([0], dtype=np.uint32))
    else:
        g = gg.rmat(9, 7, seed=3)
    if case == "caller_index":
        eo, ei = oracle.edge_index(g, 32)
        rows = [list(ei[eo[u]:eo[u + 1]]) for u in range(g.V)]
        rows = [r + r[:1] if len(r) % 3 == 1 else r for r in rows]  # some duplicates
        eo2 = np.zeros(g.V + 1, dtype=np.uint32)
        eo2[1:] = np.cumsum([len(r) for r in rows])
        ei2 = np.array([x for r in rows for x in r], dtype=np.uint32)
        h = wedge.wedge_graph_create(g.V, g.E, g.offsets, g.src, None, eo2, ei2)
        G = wedge.Graph(h)
    else:
        G = graph(g, with_weights=False)
    try:
        wedge.wedge_graph_set_tuning(G.handle, edge_index=1)
        for front in (np.ones(g.V, dtype=bool), np.arange(g.V) % 3 == 0):
            got = _transform(G, front, 0)
            np.testing.assert_array_equal(got, oracle.wedge_groups_scan(g, front, 32))
        if g.E:
            out = empty_u32(g.V)
            wedge.wedge_run_bfs(G.handle, 0, out, opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE))
            np.testing.assert_array_equal(u32(out)[: g.V], oracle.bfs_push(g, 0))
    finally:
        G.close()
