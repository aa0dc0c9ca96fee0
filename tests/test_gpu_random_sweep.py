"""Seeded random sweep of graphs and run options against the oracle.

Each case draws a graph (uniform random, small R-MAT with a random skew, or
a rewired grid; sizes from a handful of vertices to ~2^15, weights from 1 to
near 2^32 so that SSSP saturates), a root, and run options (threshold and
precision from 8-edge entries to 32 * 2^7 edges, always dense / always sparse, the push/pull hybrid, synchronous
pulls), and checks BFS, SSSP and CC bit for bit and PageRank within L1 1e-6."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _gpu import empty_u32, graph, u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu

SWITCHES = [wedge.SWITCH_THRESHOLD, wedge.SWITCH_ALWAYS_DENSE, wedge.SWITCH_ALWAYS_SPARSE]


def _case(seed):
    rng = np.random.default_rng(10_000 + seed)
    kind = seed % 3
    if kind == 0:
        V = int(rng.integers(1, 30_000))
        g = gg.random_graph(V, int(rng.integers(0, 12 * V + 1)), seed=20_000 + seed)
    elif kind == 1:
        a = float(rng.uniform(0.45, 0.75))
        rest = (1.0 - a) / 0.43
        g = gg.rmat(int(rng.integers(6, 15)), int(rng.integers(1, 24)), a=a, b=0.19 * rest, c=0.19 * rest,
                    seed=30_000 + seed)
    else:
        g = gg.grid(int(rng.integers(2, 160)), float(rng.choice([0.0, 0.01, 0.2])), seed=40_000 + seed)
    wmax = int(rng.choice([1, 7, 1000, 0xFFFF_FFF0]))
    return g.with_weights(wmax), rng


def _opts(app, rng):
    o = wedge.wedge_default_opts(app)
    o.switch_mode = int(rng.choice(SWITCHES))
    o.tau_bp = int(rng.choice([0, 1, 100, 2000, 10000]))
    o.log2_coarsen = int(rng.integers(-2, 8)) & 0xFFFFFFFF  # -1 / -2: entries of 16 / 8 edges
    mode = int(rng.integers(0, 3)) if app != "bfs" else int(rng.integers(0, 2))
    if mode == 1:
        o.sparse_push = 1
    elif mode == 2:
        o.synchronous = 1
    return o


@pytest.mark.parametrize("seed", range(96))
def test_random_graph_and_options(seed):
    g, rng = _case(seed)
    root = int(rng.integers(0, g.V))
    G = graph(g)
    try:
        out = empty_u32(g.V)
        o = _opts("bfs", rng)
        wedge.wedge_run_bfs(G.handle, root, out, o)
        np.testing.assert_array_equal(u32(out)[: g.V], oracle.bfs_push(g, root), err_msg=f"bfs {seed}")
        o = _opts("sssp", rng)
        wedge.wedge_run_sssp(G.handle, root, out, o)
        np.testing.assert_array_equal(u32(out)[: g.V], oracle.sssp_dijkstra(g, root), err_msg=f"sssp {seed}")
        if seed % 4 == 0:
            rank = torch.empty(g.V, dtype=torch.float32, device="cuda")
            wedge.wedge_run_pr(G.handle, rank, 20, 0.85)
            assert np.abs(rank.cpu().numpy() - oracle.pr_pull(g, 0.85, 20)).sum() <= 1e-6
    finally:
        G.close()
    s = gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))
    S = graph(s, with_weights=False)
    try:
        out = empty_u32(s.V)
        wedge.wedge_run_cc(S.handle, out, _opts("cc", rng))
        np.testing.assert_array_equal(u32(out)[: s.V], oracle.cc_union_find(s), err_msg=f"cc {seed}")
    finally:
        S.close()
