"""Batched BFS (one persistent launch, 64-bit query masks): every query's
levels equal the oracle's single-root BFS, bit for bit, under every policy;
the uneven batch of block-diagonal graphs gives each graph its own BFS."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _gpu import INF, graph, opts
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu


def _levels(G, V, roots, rq, Q, o=None):
    lv = torch.empty(V * Q, dtype=torch.int32, device="cuda")
    st = wedge.wedge_run_bfs_batch(G.handle, roots, rq, Q, lv, o)
    return lv.cpu().numpy().view(np.uint32).reshape(V, Q), st


@pytest.fixture(scope="module")
def g15():
    return gg.rmat(15, 16)


@pytest.fixture(scope="module")
def g15_dev(g15):
    G = graph(g15, with_weights=False)
    yield G
    G.close()


@pytest.mark.parametrize("mode", ["default", "dense", "sparse0", "sparse3"])
def test_64_roots_match_single_bfs(g15, g15_dev, mode):
    roots = gg.roots(g15, 63, seed=5)
    roots = np.append(roots, np.flatnonzero(g15.outdeg() == 0)[:1]).astype(np.uint32)  # one root without out-edges
    o = {"default": opts("bfs"), "dense": opts("bfs", switch=wedge.SWITCH_ALWAYS_DENSE),
         "sparse0": opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0),
         "sparse3": opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=3)}[mode]
    lv, st = _levels(g15_dev, g15.V, roots, None, 64, o)
    for q, r in enumerate(roots):
        np.testing.assert_array_equal(lv[:, q], oracle.bfs_push(g15, int(r)), err_msg=f"query {q}")
    assert st.iters >= 1


def test_few_queries_shared_roots_and_repeat(g15, g15_dev):
    roots = np.array([0, 17, 17, 4000, 9], dtype=np.uint32)
    rq = np.array([0, 1, 2, 2, 0], dtype=np.uint32)
    for _ in range(2):  # the captured graph is replayed
        lv, _ = _levels(g15_dev, g15.V, roots, rq, 3)
        d0 = np.minimum(oracle.bfs_push(g15, 0), oracle.bfs_push(g15, 9))
        d2 = np.minimum(oracle.bfs_push(g15, 17), oracle.bfs_push(g15, 4000))
        np.testing.assert_array_equal(lv[:, 0], d0)
        np.testing.assert_array_equal(lv[:, 1], oracle.bfs_push(g15, 17))
        np.testing.assert_array_equal(lv[:, 2], d2)


def test_uneven_batch_of_graphs():
    graphs = [gg.rmat(8 + (i % 5), 8, seed=300 + i) for i in range(40)]
    big, base = gg.block_diagonal(graphs)
    G = graph(big, with_weights=False)
    try:
        roots = base.astype(np.uint32)          # vertex 0 of every graph
        rq = (np.arange(len(graphs)) % 64).astype(np.uint32)
        lv, _ = _levels(G, big.V, roots, rq, 64)
        for i, g in enumerate(graphs):
            got = lv[base[i]:base[i] + g.V, i % 64]
            np.testing.assert_array_equal(got, oracle.bfs_push(g, 0), err_msg=f"graph {i}")
    finally:
        G.close()


def test_invalid_batches_are_rejected(g15_dev):
    lv = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_run_bfs_batch(g15_dev.handle, [1 << 20], None, 1, lv)
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_run_bfs_batch(g15_dev.handle, [0, 1], [0, 5], 2, lv)
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_run_bfs_batch(g15_dev.handle, [0], None, 65, lv)


# ---- batched SSSP: every query's distances equal Dijkstra's -------------
def _dists(G, V, roots, rq, Q, o=None):
    d = torch.empty(V * Q, dtype=torch.int32, device="cuda")
    st = wedge.wedge_run_sssp_batch(G.handle, roots, rq, Q, d, o)
    return d.cpu().numpy().view(np.uint32).reshape(V, Q), st


@pytest.fixture(scope="module")
def g15w():
    return gg.rmat(15, 16, seed=21).with_weights(255)


@pytest.fixture(scope="module")
def g15w_dev(g15w):
    G = graph(g15w)
    yield G
    G.close()


@pytest.mark.parametrize("mode", ["default", "dense", "sparse0", "sparse3"])
def test_sssp_batch_matches_dijkstra(g15w, g15w_dev, mode):
    roots = gg.roots(g15w, 64, seed=6)
    o = {"default": opts("sssp"), "dense": opts("sssp", switch=wedge.SWITCH_ALWAYS_DENSE),
         "sparse0": opts("sssp", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0),
         "sparse3": opts("sssp", switch=wedge.SWITCH_ALWAYS_SPARSE, k=3)}[mode]
    d, st = _dists(g15w_dev, g15w.V, roots, None, 64, o)
    for q in range(0, 64, 7 if mode != "default" else 1):
        np.testing.assert_array_equal(d[:, q], oracle.sssp_dijkstra(g15w, int(roots[q])), err_msg=f"query {q}")
    assert st.iters >= 1


@pytest.mark.parametrize("Q", [1, 5, 33])
def test_sssp_batch_query_counts_and_shared_roots(g15w, g15w_dev, Q):
    # Q = 33 uses the second lane half (queries 32..63); several roots per query
    rng = np.random.default_rng(Q)
    roots = gg.roots(g15w, 2 * Q, seed=40 + Q)
    rq = np.concatenate([np.arange(Q), rng.integers(0, Q, Q)]).astype(np.uint32)
    for _ in range(2):  # the captured graph is replayed
        d, _ = _dists(g15w_dev, g15w.V, roots, rq, Q)
        for q in sorted({0, Q - 1, Q // 2}):
            want = np.full(g15w.V, 0xFFFFFFFF, dtype=np.uint32)
            for r in roots[rq == q]:
                want = np.minimum(want, oracle.sssp_dijkstra(g15w, int(r)))
            np.testing.assert_array_equal(d[:, q], want, err_msg=f"Q={Q} query {q}")


def test_sssp_uneven_batch_of_graphs():
    graphs = [gg.rmat(8 + (i % 5), 8, seed=500 + i).with_weights(255) for i in range(40)]
    big, base = gg.block_diagonal(graphs)
    G = graph(big)
    try:
        d, _ = _dists(G, big.V, base.astype(np.uint32), (np.arange(len(graphs)) % 64).astype(np.uint32), 64)
        for i, g in enumerate(graphs):
            np.testing.assert_array_equal(d[base[i]:base[i] + g.V, i % 64], oracle.sssp_dijkstra(g, 0),
                                          err_msg=f"graph {i}")
    finally:
        G.close()


def test_sssp_batch_needs_weights(g15_dev):
    d = torch.empty(g15_dev.V * 2, dtype=torch.int32, device="cuda")
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_run_sssp_batch(g15_dev.handle, [0, 1], None, 2, d)


def _levels8(G, V, roots, rq, Q, o=None):
    lv = torch.empty(V * Q, dtype=torch.uint8, device="cuda")
    st = wedge.wedge_run_bfs_batch_u8(G.handle, roots, rq, Q, lv, o)
    return lv.cpu().numpy().reshape(V, Q), st


def _as_u8(levels32):
    return np.where(levels32 == INF, 0xFF, levels32).astype(np.uint8)


@pytest.mark.parametrize("mode", ["default", "sparse0", "dense"])
def test_u8_levels_equal_u32_levels(g15, g15_dev, mode):
    roots = gg.roots(g15, 64, seed=11).astype(np.uint32)
    o = {"default": opts("bfs"), "dense": opts("bfs", switch=wedge.SWITCH_ALWAYS_DENSE),
         "sparse0": opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0)}[mode]
    l8, st8 = _levels8(g15_dev, g15.V, roots, None, 64, o)
    l32, st32 = _levels(g15_dev, g15.V, roots, None, 64, o)
    np.testing.assert_array_equal(l8, _as_u8(l32))
    for q in (0, 31, 63):
        np.testing.assert_array_equal(l8[:, q], _as_u8(oracle.bfs_push(g15, int(roots[q]))))
    assert st8.iters == st32.iters
    # the 32-bit and 8-bit runs replay their own captured graphs
    l8b, _ = _levels8(g15_dev, g15.V, roots, None, 64, o)
    np.testing.assert_array_equal(l8b, l8)


def test_u8_uneven_batch():
    graphs = [gg.rmat(8 + (i % 4), 8, seed=300 + i) for i in range(20)]
    big, base = gg.block_diagonal(graphs)
    G = graph(big, with_weights=False)
    try:
        rq = (np.arange(20) % 7).astype(np.uint32)
        l8, _ = _levels8(G, big.V, base.astype(np.uint32), rq, 7)
        l32, _ = _levels(G, big.V, base.astype(np.uint32), rq, 7)
        np.testing.assert_array_equal(l8, _as_u8(l32))
    finally:
        G.close()


@pytest.mark.parametrize("n,fits", [(255, True), (300, False)])
def test_u8_levels_checked_against_255(n, fits):
    """A directed path of n vertices: levels 0 .. n-1.  Up to level 254 the
    8-bit call returns them; a level of 255 or more makes it stop and
    report that the levels do not fit (the levels it wrote are exact)."""
    g = gg.from_edges(n, list(range(n - 1)), list(range(1, n)))
    G = graph(g, with_weights=False)
    try:
        want = np.arange(n, dtype=np.int64)
        if fits:
            l8, _ = _levels8(G, n, np.array([0], dtype=np.uint32), None, 1)
            np.testing.assert_array_equal(l8[:, 0], want.astype(np.uint8))
        else:
            lv = torch.empty(n, dtype=torch.uint8, device="cuda")
            with pytest.raises(wedge.WedgeError) as e:
                wedge.wedge_run_bfs_batch_u8(G.handle, np.array([0], dtype=np.uint32), None, 1, lv)
            assert e.value.status == 5  # NOT_SUPPORTED
            got = lv.cpu().numpy()
            np.testing.assert_array_equal(got[:255], want[:255].astype(np.uint8))
            assert np.all(got[255:] == 0xFF)
            l32, _ = _levels(G, n, np.array([0], dtype=np.uint32), None, 1)
            np.testing.assert_array_equal(l32[:, 0], want.astype(np.uint32))
    finally:
        G.close()
