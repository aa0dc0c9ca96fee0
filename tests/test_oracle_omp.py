"""The oracle's all-cores timing variants (the CPU baseline's multi-threaded
leg) compute exactly what the single-threaded oracle computes: BFS, CC and
SSSP values and pull counts of dense pulls, and PageRank bit for bit (each
destination's sum keeps its CSC order)."""
import numpy as np
import pytest

import graphgen as gg
import oracle


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dense_pulls_equal_single_threaded(seed):
    g = gg.rmat(11 + seed, 8, seed=seed).with_weights(1000)
    s = gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))
    for app, h, root in (("bfs", g, 0), ("sssp", g, 0), ("cc", s, 0)):
        want, tr = oracle.wedge_run(app, h, root, oracle.POLICY_ALWAYS_DENSE)
        got, pulls = oracle.dense_pull_omp(app, h, root)
        np.testing.assert_array_equal(got, want, err_msg=app)
        assert pulls == tr.shape[0], app
    np.testing.assert_array_equal(oracle.dense_pull_omp("bfs", g, 0)[0], oracle.bfs_push(g, 0))
    np.testing.assert_array_equal(oracle.dense_pull_omp("sssp", g, 0)[0], oracle.sssp_dijkstra(g, 0))
    np.testing.assert_array_equal(oracle.dense_pull_omp("cc", s)[0], oracle.cc_union_find(s))


def test_pagerank_equals_single_threaded_bit_for_bit():
    g = gg.rmat(13, 8, seed=4)
    a = oracle.pr_pull(g, 0.85, 20)
    b = oracle.pr_pull_omp(g, 0.85, 20)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_thread_count_is_reported():
    assert oracle.omp_threads() >= 1
