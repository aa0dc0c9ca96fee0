"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Integer results (levels, labels, distances, chunk lists, edge index,
fullness, frontier sizes) must match bit for bit; PageRank (FP32) must be
within an L1 distance of 1e-6 of the FP64 oracle.  Graphs span many 128-edge
tiles and have ragged tails (E not a multiple of 4 or 32)."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _gpu import INF, bitmap, dev_u32, empty_u32, graph, opts, u32, unpack, zeros_u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu

PR_L1_TOL = 1e-6


@pytest.fixture(scope="module")
def rmat():
    """R-MAT scale 16, edge factor 16 (a=0.57, b=c=0.19) with weights in [1,255]."""
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


def _run(G, app, root=0, o=None):
    out = empty_u32(G.V)
    if app == "bfs":
        st = wedge.wedge_run_bfs(G.handle, root, out, o)
    elif app == "cc":
        st = wedge.wedge_run_cc(G.handle, out, o)
    else:
        st = wedge.wedge_run_sssp(G.handle, root, out, o)
    return u32(out)[: G.V], st


def test_edge_index_matches_oracle(rmat, rmat_dev):
    G = rmat_dev
    info = G.info
    eo = empty_u32(G.V + 1)
    ei = empty_u32(info["eidx_len"])
    wedge.wedge_graph_copy_edge_index(G.handle, eo, ei)
    eo_g, ei_g = u32(eo)[: G.V + 1].astype(np.uint64), u32(ei)[: info["eidx_len"]].astype(np.uint64)
    eo_o, ei_o = oracle.edge_index(rmat, 32)
    np.testing.assert_array_equal(eo_g, eo_o)
    rows = np.repeat(np.arange(G.V, dtype=np.uint64), np.diff(eo_g).astype(np.int64))
    order = np.lexsort((ei_g, rows))  # rows keep any order on the GPU: compare as sets
    np.testing.assert_array_equal(ei_g[order], ei_o)
    assert info["nchunks"] == (rmat.E + 31) // 32
    assert info["nz_dst"] == int((rmat.indeg() > 0).sum())


@pytest.mark.parametrize("frac", [0.0001, 0.003, 0.05, 0.6])
def test_transform_matches_definition(rmat, rmat_dev, frac):
    G = rmat_dev
    r = np.array([gg.rand(77, i) for i in range(G.V)], dtype=np.uint64)
    front = (r % np.uint64(100000)) < np.uint64(int(frac * 100000))
    front[0] = True
    bm = dev_u32(bitmap(G.V, front))
    nc = G.info["nchunks"]
    for k in (0, 1, 2, 3, 4, 7):
        cap = (nc + (1 << k) - 1) >> k
        lst = empty_u32(cap)
        cnt = zeros_u32(1)
        wedge.wedge_frontier_transform(G.handle, bm, k, lst, cnt)
        n = int(u32(cnt)[0])
        got = u32(lst)[:n].astype(np.uint64)
        assert np.unique(got).size == n, "entries must be distinct"
        want = oracle.wedge_groups_scan(rmat, front, 32 << k)
        np.testing.assert_array_equal(np.sort(got), want)


def test_transform_flushes_several_times_per_warp():
    """A frontier large enough that each transformation warp stages more than
    one batch of fresh entries (R-MAT s20, 30% of the vertices, k = 0: about
    5 M edge-index entries over the warps), so the mid-task flushes of the
    staged list are compared with the Wedge Frontier's definition too."""
    g = gg.rmat(20, 16)
    r = np.array([gg.rand(78, i) for i in range(g.V)], dtype=np.uint64)
    front = (r % np.uint64(100)) < np.uint64(30)
    G = graph(g, with_weights=False)
    try:
        bm = dev_u32(bitmap(G.V, front))
        nc = G.info["nchunks"]
        for k in (0, 1):
            cap = (nc + (1 << k) - 1) >> k
            lst = empty_u32(cap)
            cnt = zeros_u32(1)
            wedge.wedge_frontier_transform(G.handle, bm, k, lst, cnt)
            n = int(u32(cnt)[0])
            got = np.sort(u32(lst)[:n].astype(np.uint64))
            want = oracle.wedge_groups_scan(g, front, 32 << k)
            assert n == want.size
            assert np.unique(got).size == n
            np.testing.assert_array_equal(got, want)
    finally:
        G.close()


@pytest.mark.parametrize("schedule", [0, 1])
def test_transform_profile_schedules_match_definition(rmat, rmat_dev, schedule):
    """The load-balance study's transformation (the library's schedule and
    the paper's static slices) produces the Wedge Frontier's definition, and
    every warp's records are well formed: start <= end within the kernel's
    span, busy cycles > 0, an SM id below the SM count."""
    G = rmat_dev
    r = np.array([gg.rand(79, i) for i in range(G.V)], dtype=np.uint64)
    front = (r % np.uint64(100)) < np.uint64(20)
    front[0] = True          # the hub: one long row
    bm = dev_u32(bitmap(G.V, front))
    nc = G.info["nchunks"]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for k in (0, 2):
        cap = (nc + (1 << k) - 1) >> k
        lst = empty_u32(cap)
        cnt = zeros_u32(1)
        rec = wedge.wedge_frontier_transform_profile(G.handle, bm, k, schedule, lst, cnt)
        n = int(u32(cnt)[0])
        got = np.sort(u32(lst)[:n].astype(np.uint64))
        np.testing.assert_array_equal(got, oracle.wedge_groups_scan(rmat, front, 32 << k))
        kernels = (0, 1) if schedule == 0 else (0,)
        for kk in kernels:
            st, en, cyc, sm = (rec[:, kk, i] for i in range(4))
            assert np.all(st > 0) and np.all(en >= st)
            assert np.all(cyc > 0) and np.all(sm < sms)
        if schedule == 1:
            assert np.all(rec[:, 1, :] == 0)
        # the library's transformation afterwards still matches (Wedge bitmap left clear)
        cnt2 = zeros_u32(1)
        wedge.wedge_frontier_transform(G.handle, bm, k, lst, cnt2)
        n2 = int(u32(cnt2)[0])
        np.testing.assert_array_equal(np.sort(u32(lst)[:n2].astype(np.uint64)), got)


@pytest.mark.parametrize("mode", ["default", "dense", "sparse0", "sparse2", "sparse5", "tau20k1"])
def test_bfs_matches_oracle(rmat, rmat_dev, mode):
    want = oracle.bfs_push(rmat, 0)
    o = {"default": opts("bfs"), "dense": opts("bfs", switch=wedge.SWITCH_ALWAYS_DENSE),
         "sparse0": opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0),
         "sparse2": opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=2),
         "sparse5": opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=5),
         "tau20k1": opts("bfs", tau=2000, k=1)}[mode]
    got, st = _run(rmat_dev, "bfs", 0, o)
    np.testing.assert_array_equal(got, want)
    assert st.iters == int(want[want != INF].max()) + 1


@pytest.mark.parametrize("tau,k", [(100, 3), (2000, 0), (500, 2)])
def test_bfs_trace_matches_oracle(rmat, rmat_dev, tau, k):
    """BFS is level-synchronous on both sides, so every iteration's frontier
    size, fullness, decision and Wedge Frontier size must agree."""
    o = opts("bfs", tau=tau, k=k, trace=1)
    got, st = _run(rmat_dev, "bfs", 0, o)
    tr = wedge.wedge_get_trace(rmat_dev.handle)
    _, ot = oracle.wedge_run("bfs", rmat, 0, oracle.POLICY_THRESHOLD, tau, 32 << k)
    assert len(tr) == ot.shape[0] == st.iters
    for t, rec in enumerate(tr):
        assert rec["nfront"] == ot[t, 0], t
        assert rec["fullness"] == ot[t, 1], t
        assert rec["mode"] == ot[t, 2], t
        if rec["mode"]:
            assert rec["nchunks"] == ot[t, 3], t


@pytest.mark.parametrize("app", ["cc", "sssp"])
@pytest.mark.parametrize("policy,tau,k", [("threshold", 2000, 2), ("threshold", 500, 0), ("threshold", 5000, 1),
                                          ("sparse", 0, 3), ("dense", 0, 0)])
def test_synchronous_trace_matches_oracle(rmat, rmat_dev, sym, sym_dev, app, policy, tau, k):
    """Synchronous CC/SSSP (every pull reads the previous iteration's values,
    as the oracle's Wedge run does): every iteration's frontier size,
    fullness, decision and Wedge Frontier size agree, and so do the values
    and the iteration count."""
    g, G = (sym, sym_dev) if app == "cc" else (rmat, rmat_dev)
    sw = {"threshold": None, "sparse": wedge.SWITCH_ALWAYS_SPARSE, "dense": wedge.SWITCH_ALWAYS_DENSE}[policy]
    pol = {"threshold": oracle.POLICY_THRESHOLD, "sparse": oracle.POLICY_ALWAYS_SPARSE,
           "dense": oracle.POLICY_ALWAYS_DENSE}[policy]
    o = opts(app, switch=sw, tau=tau, k=k, trace=1)
    o.synchronous = 1
    got, st = _run(G, app, 0, o)
    tr = wedge.wedge_get_trace(G.handle)
    want, ot = oracle.wedge_run(app, g, 0, pol, tau, 32 << k)
    np.testing.assert_array_equal(got, want)
    assert len(tr) == ot.shape[0] == st.iters
    for t, rec in enumerate(tr):
        assert rec["nfront"] == ot[t, 0], t
        assert rec["fullness"] == ot[t, 1], t
        assert rec["mode"] == ot[t, 2], t
        if rec["mode"]:
            assert rec["nchunks"] == ot[t, 3], t
    # untraced (the loop without records) ends the same way
    o.trace = 0
    got2, st2 = _run(G, app, 0, o)
    np.testing.assert_array_equal(got2, want)
    assert st2.iters == st.iters


@pytest.mark.parametrize("mode", ["default", "dense", "sparse0", "sparse3", "tau50k1"])
def test_cc_matches_union_find(sym, sym_dev, mode):
    want = oracle.cc_union_find(sym)
    o = {"default": opts("cc"), "dense": opts("cc", switch=wedge.SWITCH_ALWAYS_DENSE),
         "sparse0": opts("cc", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0),
         "sparse3": opts("cc", switch=wedge.SWITCH_ALWAYS_SPARSE, k=3),
         "tau50k1": opts("cc", tau=5000, k=1)}[mode]
    got, _ = _run(sym_dev, "cc", 0, o)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("mode", ["default", "dense", "sparse0", "sparse4"])
def test_sssp_matches_dijkstra(rmat, rmat_dev, mode):
    want = oracle.sssp_dijkstra(rmat, 0)
    o = {"default": opts("sssp"), "dense": opts("sssp", switch=wedge.SWITCH_ALWAYS_DENSE),
         "sparse0": opts("sssp", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0),
         "sparse4": opts("sssp", switch=wedge.SWITCH_ALWAYS_SPARSE, k=4)}[mode]
    got, _ = _run(rmat_dev, "sssp", 0, o)
    np.testing.assert_array_equal(got, want)


def test_pagerank_l1(rmat, rmat_dev):
    want = oracle.pr_pull(rmat, 0.85, 20)
    rank = torch.empty(rmat.V, dtype=torch.float32, device="cuda")
    wedge.wedge_run_pr(rmat_dev.handle, rank, 20, 0.85)
    got = rank.cpu().numpy().astype(np.float64)
    l1 = np.abs(got - want).sum()
    assert l1 <= PR_L1_TOL, l1
    # the exact fixed-point sums make the result independent of the schedule
    rank2 = torch.empty_like(rank)
    wedge.wedge_run_pr(rmat_dev.handle, rank2, 20, 0.85)
    assert torch.equal(rank, rank2)


@pytest.mark.parametrize("which", ["rmat", "sym"])
def test_pr_pull_in_sums(rmat, rmat_dev, sym, sym_dev, which):
    """PageRank's in-edge pass alone: the exact 2^-62 fixed-point sums
    against the oracle's FP64 in-edge sums of the same FP32 values; a sum of
    n terms differs by at most n/2 units of 2^-62 plus FP64 rounding."""
    g, G = (rmat, rmat_dev) if which == "rmat" else (sym, sym_dev)
    x = (np.random.default_rng(7).random(g.V) / g.V).astype(np.float32)
    sums = torch.zeros(g.V, dtype=torch.int64, device="cuda")
    wedge.wedge_pr_pull(G.handle, torch.from_numpy(x).cuda(), sums)
    got = sums.cpu().numpy().view(np.uint64)
    want = oracle.in_sums(g, x.astype(np.float64))
    indeg = np.diff(g.offsets.astype(np.int64))
    err = np.abs(got.astype(np.float64) * 2.0**-62 - want)
    assert np.all(err <= (indeg + 1) * 2.0**-62 + 4e-16 * want), err.max()
    assert np.all(got[indeg == 0] == 0)
    # same values, same sums: the schedule does not show
    again = torch.zeros_like(sums)
    wedge.wedge_pr_pull(G.handle, torch.from_numpy(x).cuda(), again)
    assert torch.equal(sums, again)


@pytest.mark.parametrize("which", ["rmat", "sym"])
def test_pr_gather_order(rmat, rmat_dev, sym, sym_dev, which):
    """PageRank gathers contributions stored by rank of descending
    out-degree (ties by id): the exported order is that ranking, and the
    pull on contributions placed by it gives the by-vertex pull's exact
    sums."""
    g, G = (rmat, rmat_dev) if which == "rmat" else (sym, sym_dev)
    order = torch.empty(g.V, dtype=torch.int32, device="cuda")
    wedge.wedge_pr_order(G.handle, order)
    got = order.cpu().numpy().astype(np.int64)
    rank = np.empty(g.V, dtype=np.int64)
    rank[np.argsort(-g.outdeg().astype(np.int64), kind="stable")] = np.arange(g.V)
    np.testing.assert_array_equal(got, rank)
    x = (np.random.default_rng(8).random(g.V) / g.V).astype(np.float32)
    xo = np.empty_like(x)
    xo[got] = x
    a = torch.zeros(g.V, dtype=torch.int64, device="cuda")
    b = torch.zeros_like(a)
    wedge.wedge_pr_pull(G.handle, torch.from_numpy(x).cuda(), a)
    wedge.wedge_pr_pull_ordered(G.handle, torch.from_numpy(xo).cuda(), b)
    assert torch.equal(a, b)


def test_pull_iterate_bfs_step(rmat, rmat_dev):
    """One BFS iteration from the oracle's level-t state, dense and over the
    Wedge Frontier, yields exactly the level-(t+1) set."""
    G = rmat_dev
    lvl = oracle.bfs_push(rmat, 0)
    od = oracle.outdeg(rmat)
    depth = int(lvl[lvl != INF].max())
    for t in range(depth):
        state = np.where(lvl <= t, lvl, INF).astype(np.uint32)
        cur = dev_u32(bitmap(G.V, lvl == t))
        for sparse in (False, True):
            vals = dev_u32(state)
            nxt = zeros_u32((G.V + 31) // 32)
            full = torch.zeros(1, dtype=torch.int64, device="cuda")
            nf = zeros_u32(1)
            lst = cnt = None
            k = 2
            if sparse:
                lst = empty_u32(G.info["nchunks"])
                cnt = zeros_u32(1)
                wedge.wedge_frontier_transform(G.handle, cur, k, lst, cnt)
            wedge.wedge_pull_iterate(G.handle, "bfs", vals, t, cur, lst, cnt, k, nxt, full, nf)
            want = np.where(lvl <= t + 1, lvl, INF).astype(np.uint32)
            np.testing.assert_array_equal(u32(vals)[: G.V], want)
            np.testing.assert_array_equal(unpack(u32(nxt), G.V), lvl == t + 1)
            assert int(full.item()) == int(od[lvl == t + 1].sum())
            assert int(u32(nf)[0]) == int((lvl == t + 1).sum())


@pytest.mark.parametrize("app", ["cc", "sssp"])
def test_pull_iterate_min_step_bounds(rmat, sym, rmat_dev, sym_dev, app):
    """CC/SSSP update in place, so one GPU iteration may move values further
    than one synchronous step; it can never overshoot the fixed point, and the
    reported frontier is exactly the set of vertices whose value dropped."""
    g, G = (sym, sym_dev) if app == "cc" else (rmat, rmat_dev)
    fixed = oracle.cc_union_find(g) if app == "cc" else oracle.sssp_dijkstra(g, 0)
    # state after two synchronous iterations from the start
    state, _ = oracle.wedge_run(app, g, 0, oracle.POLICY_ALWAYS_DENSE, 0, 32, max_iters=2)
    one, _ = oracle.wedge_run(app, g, 0, oracle.POLICY_ALWAYS_DENSE, 0, 32, max_iters=3)
    vals = dev_u32(state)
    nxt = zeros_u32((G.V + 31) // 32)
    full = torch.zeros(1, dtype=torch.int64, device="cuda")
    nf = zeros_u32(1)
    wedge.wedge_pull_iterate(G.handle, app, vals, 2, None, None, None, 0, nxt, full, nf)
    got = u32(vals)[: G.V]
    assert np.all(got <= one) and np.all(got >= fixed)
    changed = got < state
    np.testing.assert_array_equal(unpack(u32(nxt), G.V), changed)
    assert int(u32(nf)[0]) == int(changed.sum())
    assert int(full.item()) == int(oracle.outdeg(g)[changed].sum())


def _small_cases():
    cases = []
    for i, (V, m) in enumerate([(1, 0), (7, 0), (5, 3), (40, 37), (64, 130), (300, 1201), (1000, 3333),
                                (4096, 70001)]):
        cases.append(gg.random_graph(V, m, seed=900 + i))
    cases.append(gg.grid(64, 0.0))
    cases.append(gg.grid(48, 0.02))
    return cases


@pytest.mark.parametrize("idx", range(10))
def test_small_and_degenerate_graphs(idx):
    g = _small_cases()[idx].with_weights(1000)
    G = graph(g)
    try:
        roots = sorted({0, g.V - 1, g.V // 2})
        for root in roots:
            got, _ = _run(G, "bfs", root, opts("bfs"))
            np.testing.assert_array_equal(got, oracle.bfs_push(g, root))
            got, _ = _run(G, "sssp", root, opts("sssp", switch=wedge.SWITCH_ALWAYS_SPARSE, k=0))
            np.testing.assert_array_equal(got, oracle.sssp_dijkstra(g, root))
        s = gg.symmetrize(g)
        Gs = graph(s, with_weights=False)
        got, _ = _run(Gs, "cc", 0, opts("cc"))
        np.testing.assert_array_equal(got, oracle.cc_union_find(s))
        Gs.close()
        rank = torch.empty(g.V, dtype=torch.float32, device="cuda")
        wedge.wedge_run_pr(G.handle, rank, 20, 0.85)
        assert np.abs(rank.cpu().numpy() - oracle.pr_pull(g, 0.85, 20)).sum() <= PR_L1_TOL
    finally:
        G.close()


def test_graphs_reuse_pooled_memory_and_trim():
    """Graph memory comes from the library's pool: create/destroy cycles and
    a trim in between leave every run exact."""
    g = gg.rmat(12, 8, seed=11).with_weights(255)
    want = oracle.sssp_dijkstra(g, 0)
    for i in range(4):
        G = graph(g)
        try:
            got, _ = _run(G, "sssp", 0, opts("sssp"))
            np.testing.assert_array_equal(got, want)
        finally:
            G.close()
        if i == 1:
            wedge.wedge_trim_memory(-1)
    wedge.wedge_trim_memory(0)
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_trim_memory(-2)


def test_host_buffers_and_caller_edge_index():
    """Host (numpy) CSC and outputs go through the same entry points; a
    caller-supplied edge index gives the same results as the built one."""
    g = gg.rmat(12, 16).with_weights(255)
    h = wedge.wedge_graph_create(g.V, g.E, g.offsets, g.src, g.w)
    try:
        out = np.empty(g.V, dtype=np.uint32)
        wedge.wedge_run_bfs(h, 0, out)
        np.testing.assert_array_equal(out, oracle.bfs_push(g, 0))
        wedge.wedge_run_sssp(h, 0, out)
        np.testing.assert_array_equal(out, oracle.sssp_dijkstra(g, 0))
    finally:
        wedge.wedge_graph_destroy(h)
    eo, ei = oracle.edge_index(g, 32)
    h = wedge.wedge_graph_create(g.V, g.E, g.offsets, g.src, g.w, eo.astype(np.uint32), ei.astype(np.uint32))
    try:
        out = np.empty(g.V, dtype=np.uint32)
        wedge.wedge_run_bfs(h, 0, out, opts("bfs", switch=wedge.SWITCH_ALWAYS_SPARSE, k=1))
        np.testing.assert_array_equal(out, oracle.bfs_push(g, 0))
    finally:
        wedge.wedge_graph_destroy(h)


def test_invalid_arguments_are_rejected():
    g = gg.rmat(8, 4)
    bad = g.src.copy()
    bad[5] = g.V  # out-of-range source id: caught by the device-side check
    with pytest.raises(wedge.WedgeError) as e:
        wedge.wedge_graph_create(g.V, g.E, g.offsets, bad)
    assert e.value.status == 1
    off = g.offsets.copy()
    i = int(np.flatnonzero(off[: g.V - 1] > 0)[0])
    off[i + 1] = off[i] - 1  # decreasing offsets, still 0 .. E at the ends
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_graph_create(g.V, g.E, off, g.src)
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_graph_create(g.V, g.E, g.offsets, g.src, chunk_edges=64)
    G = graph(g, with_weights=False)
    try:
        out = empty_u32(g.V)
        with pytest.raises(wedge.WedgeError):
            wedge.wedge_run_bfs(G.handle, g.V, out)
        with pytest.raises(wedge.WedgeError):
            wedge.wedge_run_sssp(G.handle, 0, out)  # no weights
        o = opts("bfs")
        o.log2_coarsen = 9
        with pytest.raises(wedge.WedgeError):
            wedge.wedge_run_bfs(G.handle, 0, out, o)
        o = opts("bfs", max_iters=1)
        with pytest.raises(wedge.WedgeError) as e:
            wedge.wedge_run_bfs(G.handle, 0, out, o)
        assert e.value.status == 6
    finally:
        G.close()


def _short_segments():
    """Every destination has one or two in-edges, so a 256-edge pull slice
    holds 170-256 destination segments: more records than a warp buffers at
    once, applied in several passes."""
    V = 50_000
    v = np.arange(V, dtype=np.int64)
    src = np.concatenate([(v * 7919 + 1) % V, ((v * 31 + 5) % V)[v % 3 == 0]])
    dst = np.concatenate([v, v[v % 3 == 0]])
    return gg.from_edges(V, src, dst).with_weights(1000)


@pytest.mark.parametrize("switch", [wedge.SWITCH_ALWAYS_DENSE, wedge.SWITCH_ALWAYS_SPARSE, None])
def test_many_short_segments(switch):
    g = _short_segments()
    assert g.src.size > 60_000
    G = graph(g)
    try:
        for root in (0, 12345):
            got, _ = _run(G, "bfs", root, opts("bfs", switch=switch))
            np.testing.assert_array_equal(got, oracle.bfs_push(g, root))
            got, _ = _run(G, "sssp", root, opts("sssp", switch=switch, k=1))
            np.testing.assert_array_equal(got, oracle.sssp_dijkstra(g, root))
        rank = torch.empty(g.V, dtype=torch.float32, device="cuda")
        wedge.wedge_run_pr(G.handle, rank, 20, 0.85)
        assert np.abs(rank.cpu().numpy() - oracle.pr_pull(g, 0.85, 20)).sum() <= PR_L1_TOL
    finally:
        G.close()
    s = gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))
    S = graph(s, with_weights=False)
    try:
        got, _ = _run(S, "cc", 0, opts("cc", switch=switch))
        np.testing.assert_array_equal(got, oracle.cc_union_find(s))
    finally:
        S.close()


@pytest.mark.parametrize("cut", [0, 5, 301])
def test_gather_probe_sums_the_gathered_values(rmat, cut):
    """The benchmark's probe (libwedge_probe.so) gathers vals[src] once per
    edge: with integer-valued floats the sum is exact, sum over the edges'
    sources of vals[u] (a ragged tail when `cut` edges are left off)."""
    from paper_1903_07754_gb300 import probe
    E = rmat.E - cut
    src = dev_u32(rmat.src[:E])
    vals = torch.from_numpy((np.arange(rmat.V) % 3).astype(np.float32)).cuda()
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    probe.wedge_probe_gather(src, E, vals, sink)
    want = float((rmat.src[:E].astype(np.int64) % 3).sum())
    assert want < 2 ** 24
    assert float(sink.item()) == want
