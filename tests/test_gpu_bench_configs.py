"""Parity at the full sizes of the benchmark's other configurations, in the
launch configuration `bench.py` times, checked on the GPU by the equations
that define the result (the oracle would take minutes per root here).

BFS levels and SSSP distances from a root are the unique solution of
Bellman's equations: d(root) = 0 and, for every other vertex,
d(v) = min over in-edges (u, v) of d(u) + w(u, v) (w = 1 for BFS), with
unreached vertices (and additions past the saturation value) at
0xFFFFFFFF / 0xFFFFFFFE as the engine defines them.  Checking every vertex's
equation therefore checks the whole output exactly.
Workloads: R-MAT scale 24 with the learned switch (BFS, SSSP), the rewired
4096^2 grid (BFS, SSSP), R-MAT scale 26 batched BFS and SSSP (64 roots, two
queries of each checked; and three of the sixteen 64-root waves of the
1024-root run with the benchmark's autotuned settings, two queries of each),
and the uneven batch of 256 R-MAT graphs of scales 12-20 (every query)."""
import numpy as np
import pytest
import torch

import graphgen as gg
from _gpu import graph, opts
from paper_1903_07754_gb300 import costmodel, wedge

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF
SAT = 0xFFFFFFFE


def _edges(g):
    """(dst, src) per CSC position as int64 CUDA tensors."""
    off = torch.from_numpy(g.offsets.astype(np.int64)).cuda()
    src = torch.from_numpy(g.src.astype(np.int64)).cuda()
    dst = torch.repeat_interleave(torch.arange(g.V, device="cuda"), off[1:] - off[:-1])
    return dst, src


def _bellman(dst, src, w, V, root, d):
    """Asserts d (int64 CUDA, INF = unreached) solves Bellman's equations;
    `root` is one vertex or an array of them (a query with several roots:
    the distance to the nearest)."""
    du = d[src]
    cand = torch.where(du == INF, torch.full_like(du, INF), torch.clamp(du + w, max=SAT))
    best = torch.full((V,), INF, dtype=torch.int64, device="cuda").scatter_reduce(
        0, dst, cand, reduce="amin", include_self=True)
    best[torch.as_tensor(np.asarray(root, dtype=np.int64), device="cuda")] = 0
    bad = int((best != d).sum().item())
    assert bad == 0, f"{bad} vertices violate the equations"
    assert int((d != INF).sum().item()) > 1


def _u32(t):
    return t.to(torch.int64) & 0xFFFFFFFF


@pytest.fixture(scope="module")
def g24():
    return gg.rmat(24, 16).with_weights(255)


def test_learned_switch_scale24(g24):
    dst, src = _edges(g24)
    w = torch.from_numpy(g24.w.astype(np.int64)).cuda()
    G = graph(g24)
    try:
        wedge.wedge_set_cost_model(G.handle, costmodel.load_params())
        out = torch.empty(g24.V, dtype=torch.int32, device="cuda")
        st = wedge.wedge_run_bfs(G.handle, 0, out, opts("bfs", switch=wedge.SWITCH_LEARNED))
        _bellman(dst, src, torch.ones_like(w), g24.V, 0, _u32(out))
        assert st.iters > 1
        wedge.wedge_run_sssp(G.handle, 0, out, opts("sssp", switch=wedge.SWITCH_LEARNED))
        _bellman(dst, src, w, g24.V, 0, _u32(out))
    finally:
        G.close()


def test_rewired_grid_4096():
    g = gg.grid(4096, 0.01).with_weights(1000)
    dst, src = _edges(g)
    w = torch.from_numpy(g.w.astype(np.int64)).cuda()
    G = graph(g)
    try:
        out = torch.empty(g.V, dtype=torch.int32, device="cuda")
        wedge.wedge_run_bfs(G.handle, 0, out, opts("bfs"))
        _bellman(dst, src, torch.ones_like(w), g.V, 0, _u32(out))
        wedge.wedge_run_sssp(G.handle, 0, out, opts("sssp"))
        _bellman(dst, src, w, g.V, 0, _u32(out))
    finally:
        G.close()


@pytest.fixture(scope="module")
def g26():
    return gg.rmat(26, 16).with_weights(255)


def test_batched_bfs_and_sssp_scale26(g26):
    g = g26
    roots = gg.roots(g, 64, seed=3)
    G = graph(g)
    try:
        lv = torch.empty(g.V * 64, dtype=torch.int32, device="cuda")
        dst, src = _edges(g)
        wedge.wedge_run_bfs_batch(G.handle, roots, None, 64, lv)
        one = torch.ones(1, dtype=torch.int64, device="cuda").expand(src.numel())
        for q in (0, 37):
            _bellman(dst, src, one, g.V, int(roots[q]), _u32(lv.view(g.V, 64)[:, q].contiguous()))
        del one
        wedge.wedge_run_sssp_batch(G.handle, roots, None, 64, lv)
        w = torch.from_numpy(g.w.astype(np.int64)).cuda()
        for q in (5, 63):
            _bellman(dst, src, w, g.V, int(roots[q]), _u32(lv.view(g.V, 64)[:, q].contiguous()))
    finally:
        G.close()


def test_batched_1024_roots_scale26_waves(g26):
    """The 1024-root run as the benchmark times it: the batched-BFS settings
    its autotuner picks on the first 64 roots, then 16 waves of 64 roots;
    waves 0, 7 and 15 are checked (two queries each), for BFS and SSSP."""
    from paper_1903_07754_gb300 import autotune
    g = g26
    roots = gg.roots(g, 1024, seed=3)
    G = graph(g)
    try:
        best, _ = autotune.tune(G.handle, "bfs_batch", g.V, roots=roots[:64], nqueries=64,
                                grid={"k": (1, 2, 3), "tau_bp": (500, 2000, 5000)}, reps=1)
        autotune.apply(G.handle, best)
        o = autotune.opts_for("bfs_batch", best)
        lv = torch.empty(g.V * 64, dtype=torch.int32, device="cuda")
        dst, src = _edges(g)
        one = torch.ones(1, dtype=torch.int64, device="cuda").expand(src.numel())
        w = torch.from_numpy(g.w.astype(np.int64)).cuda()
        for wave in (0, 7, 15):
            r = roots[64 * wave:64 * (wave + 1)]
            wedge.wedge_run_bfs_batch(G.handle, r, None, 64, lv, o, False)
            for q in (wave % 64, (13 * wave + 5) % 64):
                _bellman(dst, src, one, g.V, int(r[q]), _u32(lv.view(g.V, 64)[:, q].contiguous()))
            wedge.wedge_run_sssp_batch(G.handle, r, None, 64, lv, None, False)
            for q in ((wave + 31) % 64, (7 * wave + 2) % 64):
                _bellman(dst, src, w, g.V, int(r[q]), _u32(lv.view(g.V, 64)[:, q].contiguous()))
    finally:
        G.close()


def test_uneven_batch_of_256_graphs_full_size():
    """The benchmark's uneven batch: 256 R-MAT graphs of scales 12 + (i mod 9)
    concatenated block-diagonally, graph i's vertex 0 a root of query
    i mod 64 (four graphs per query).  Every query's levels and distances
    solve Bellman's equations with its four roots."""
    graphs = [gg.rmat(12 + (i % 9), 16, seed=1000 + i).with_weights(255) for i in range(256)]
    big, base = gg.block_diagonal(graphs)
    del graphs
    rq = (np.arange(256) % 64).astype(np.uint32)
    roots = base[:256].astype(np.uint32)
    G = graph(big)
    try:
        lv = torch.empty(big.V * 64, dtype=torch.int32, device="cuda")
        dst, src = _edges(big)
        one = torch.ones(1, dtype=torch.int64, device="cuda").expand(src.numel())
        w = torch.from_numpy(big.w.astype(np.int64)).cuda()
        wedge.wedge_run_bfs_batch(G.handle, roots, rq, 64, lv, None, False)
        for q in range(64):
            _bellman(dst, src, one, big.V, roots[rq == q], _u32(lv.view(big.V, 64)[:, q].contiguous()))
        wedge.wedge_run_sssp_batch(G.handle, roots, rq, 64, lv, None, False)
        for q in range(64):
            _bellman(dst, src, w, big.V, roots[rq == q], _u32(lv.view(big.V, 64)[:, q].contiguous()))
    finally:
        G.close()


def test_more_than_2_31_edges():
    """Edge positions past 2^31 (signed 32-bit overflow territory): a
    structured graph with V = 2^26 and in-degree 32 (+ a ragged tail), built
    on the device; BFS and SSSP checked through Bellman's equations."""
    V, d, stride = 1 << 26, 32, 1 << 20
    v = torch.arange(V, device="cuda", dtype=torch.int64)
    j = torch.arange(d, device="cuda", dtype=torch.int64)
    src2 = torch.sort((v[:, None] * 3 + j[None, :] * stride + 1) % V, dim=1).values
    extra = torch.arange(5, 42, device="cuda", dtype=torch.int64)   # 37 more in-edges of the last vertex
    last = torch.unique(torch.cat([src2[-1], extra]))
    src = torch.cat([src2[:-1].reshape(-1), last]).to(torch.int32)
    deg = torch.full((V,), d, device="cuda", dtype=torch.int64)
    deg[-1] = last.numel()
    off = torch.zeros(V + 1, device="cuda", dtype=torch.int64)
    off[1:] = torch.cumsum(deg, 0)
    E = int(off[-1].item())
    assert E > 2**31
    w = ((src.to(torch.int64) * 7 + torch.repeat_interleave(v, deg)) % 13 + 1).to(torch.int32)
    off32 = off.to(torch.int32)
    del src2
    h = wedge.wedge_graph_create(V, E, off32, src, w)
    G = wedge.Graph(h, keep=[off32, src, w])
    try:
        out = torch.empty(V, dtype=torch.int32, device="cuda")
        st = wedge.wedge_run_bfs(G.handle, 0, out, opts("bfs"))
        dst = torch.repeat_interleave(v, deg)
        s64 = src.to(torch.int64)
        _bellman(dst, s64, torch.ones(1, dtype=torch.int64, device="cuda").expand(E), V, 0, _u32(out))
        assert st.iters > 2
        wedge.wedge_run_sssp(G.handle, 0, out, opts("sssp"))
        _bellman(dst, s64, w.to(torch.int64), V, 0, _u32(out))
    finally:
        G.close()
