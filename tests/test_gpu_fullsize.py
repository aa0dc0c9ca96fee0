"""Parity at the full benchmark size (R-MAT scale 22, edge factor 16), in the
launch configuration the benchmark times (default options): BFS, CC and SSSP
bit-exact against the oracle over every vertex, PageRank within L1 1e-6."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _gpu import empty_u32, graph, u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g22():
    return gg.rmat(22, 16).with_weights(255)


def test_bfs_sssp_pr_scale22(g22):
    G = graph(g22)
    try:
        out = empty_u32(g22.V)
        wedge.wedge_run_bfs(G.handle, 0, out)
        np.testing.assert_array_equal(u32(out)[: g22.V], oracle.bfs_push(g22, 0))
        wedge.wedge_run_sssp(G.handle, 0, out)
        np.testing.assert_array_equal(u32(out)[: g22.V], oracle.sssp_dijkstra(g22, 0))
        rank = torch.empty(g22.V, dtype=torch.float32, device="cuda")
        wedge.wedge_run_pr(G.handle, rank, 20, 0.85)
        l1 = np.abs(rank.cpu().numpy().astype(np.float64) - oracle.pr_pull(g22, 0.85, 20)).sum()
        assert l1 <= 1e-6, l1
    finally:
        G.close()


def test_cc_scale22(g22):
    s = gg.symmetrize(gg.Graph(g22.V, g22.offsets, g22.src))
    G = graph(s, with_weights=False)
    try:
        out = empty_u32(s.V)
        wedge.wedge_run_cc(G.handle, out)
        np.testing.assert_array_equal(u32(out)[: s.V], oracle.cc_union_find(s))
    finally:
        G.close()
