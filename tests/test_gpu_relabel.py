"""Degree-ordered relabelling (a locality step before graph creation, not in
the paper) and the calls that bring results back to the original ids.

The relabelled CSC must equal its plain definition computed here with numpy
(new ids by descending out-degree, ties by ascending old id; each
destination's in-edges in their original order with renamed sources), and
every application run on the relabelled graph, mapped back, must equal the
oracle on the original graph: BFS levels, SSSP distances and component
labels bit for bit, PageRank within the usual L1 bound and bit-identical to
the run on the original graph (its sums are exact)."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _gpu import dev_u32, empty_u32, u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu


def _definition(g):
    """(new_of_old, old_of_new, offsets, src, w) of the relabelled CSC."""
    od = np.bincount(g.src.astype(np.int64), minlength=g.V)
    old_of_new = np.argsort(-od, kind="stable")
    new_of_old = np.empty(g.V, dtype=np.int64)
    new_of_old[old_of_new] = np.arange(g.V)
    indeg = np.diff(g.offsets.astype(np.int64))[old_of_new]
    off = np.concatenate([[0], np.cumsum(indeg)]).astype(np.uint32)
    src = np.concatenate([new_of_old[g.src[g.offsets[o]:g.offsets[o + 1]].astype(np.int64)] for o in old_of_new]
                         + [np.zeros(0, dtype=np.int64)]).astype(np.uint32)
    w = None
    if g.w is not None:
        w = np.concatenate([g.w[g.offsets[o]:g.offsets[o + 1]] for o in old_of_new]
                           + [np.zeros(0, dtype=np.uint32)]).astype(np.uint32)
    return new_of_old.astype(np.uint32), old_of_new.astype(np.uint32), off, src, w


def _relabel(g):
    """Device relabelling of g: (graphgen Graph of the result, new_of_old,
    old_of_new) with the device arrays kept on the Graph."""
    off, src = dev_u32(g.offsets), dev_u32(g.src if g.E else np.zeros(4, np.uint32))
    w = dev_u32(g.w) if g.w is not None else None
    noff, nsrc = empty_u32(g.V + 1), empty_u32(max(g.E, 4))
    nw = empty_u32(max(g.E, 4)) if w is not None else None
    n2o, o2n = empty_u32(g.V), empty_u32(g.V)
    wedge.wedge_csc_relabel_by_degree(g.V, g.E, off, src, w, noff, nsrc, nw, o2n, n2o)
    torch.cuda.synchronize()
    h = gg.Graph(g.V, u32(noff)[: g.V + 1].copy(), u32(nsrc)[: g.E].copy(),
                 u32(nw)[: g.E].copy() if nw is not None else None)
    return h, o2n, n2o


@pytest.fixture(scope="module")
def rm():
    return gg.rmat(14, 16).with_weights(255)


@pytest.mark.parametrize("case", ["rmat14", "grid", "isolated", "one"])
def test_relabelled_csc_matches_definition(case, rm):
    g = {"rmat14": rm,
         "grid": gg.grid(64, 0.05).with_weights(9),
         "isolated": gg.from_edges(300, [5, 5, 5, 7, 9, 299], [7, 9, 299, 5, 5, 0]),
         "one": gg.from_edges(1, [], [])}[case]
    h, o2n, n2o = _relabel(g)
    want = _definition(g)
    np.testing.assert_array_equal(u32(o2n)[: g.V], want[0])
    np.testing.assert_array_equal(u32(n2o)[: g.V], want[1])
    np.testing.assert_array_equal(h.offsets, want[2])
    np.testing.assert_array_equal(h.src, want[3])
    if g.w is not None:
        np.testing.assert_array_equal(h.w, want[4])


def test_runs_on_relabelled_graph_match_oracle(rm):
    g = rm
    h, o2n, n2o = _relabel(g)
    G = wedge.Graph.from_csc(h)
    try:
        V = g.V
        o2n_h = u32(o2n)[:V]
        for root in (0, 1234, int(np.argmin(np.bincount(g.src.astype(np.int64), minlength=V)))):
            out, back = empty_u32(V), empty_u32(V)
            wedge.wedge_run_bfs(G.handle, int(o2n_h[root]), out)
            wedge.wedge_permute_rows(V, 1, o2n, out, back)
            np.testing.assert_array_equal(u32(back)[:V], oracle.bfs_push(g, root))
            wedge.wedge_run_sssp(G.handle, int(o2n_h[root]), out)
            wedge.wedge_permute_rows(V, 1, o2n, out, back)
            np.testing.assert_array_equal(u32(back)[:V], oracle.sssp_dijkstra(g, root))
        # PageRank: exact sums, so the relabelled run is the original run permuted
        rank = torch.empty(V, dtype=torch.float32, device="cuda")
        wedge.wedge_run_pr(G.handle, rank, 20, 0.85)
        back = torch.empty_like(rank)
        wedge.wedge_permute_rows(V, 1, o2n, rank, back)
        G0 = wedge.Graph.from_csc(g)
        r0 = torch.empty_like(rank)
        wedge.wedge_run_pr(G0.handle, r0, 20, 0.85)
        G0.close()
        np.testing.assert_array_equal(back.cpu().numpy(), r0.cpu().numpy())
        assert np.abs(back.cpu().numpy().astype(np.float64) - oracle.pr_pull(g, 0.85, 20)).sum() <= 1e-6
        # batched rows: width Q
        roots = np.array([0, 77, 4000, 9], dtype=np.uint32)
        lv, lvb = empty_u32(V * 4), empty_u32(V * 4)
        wedge.wedge_run_bfs_batch(G.handle, o2n_h[roots].astype(np.uint32), None, 4, lv)
        wedge.wedge_permute_rows(V, 4, o2n, lv, lvb)
        got = u32(lvb)[: V * 4].reshape(V, 4)
        for q, r in enumerate(roots):
            np.testing.assert_array_equal(got[:, q], oracle.bfs_push(g, int(r)))
    finally:
        G.close()


def test_cc_labels_back_to_original_ids():
    s = gg.symmetrize(gg.rmat(13, 4))
    h, o2n, n2o = _relabel(s)
    G = wedge.Graph.from_csc(h, with_weights=False)
    try:
        lab, scratch, out = empty_u32(s.V), empty_u32(s.V), empty_u32(s.V)
        wedge.wedge_run_cc(G.handle, lab)
        wedge.wedge_cc_labels_to_original(s.V, n2o, lab, scratch, out)
        np.testing.assert_array_equal(u32(out)[: s.V], oracle.cc_union_find(s))
    finally:
        G.close()


def test_relabel_rejects_bad_input(rm):
    g = rm
    off, src = dev_u32(g.offsets), dev_u32(g.src)
    noff, nsrc, o2n = empty_u32(g.V + 1), empty_u32(g.E), empty_u32(g.V)
    bad = g.src.copy()
    bad[g.E // 2] = g.V
    with pytest.raises(wedge.WedgeError, match="source id"):
        wedge.wedge_csc_relabel_by_degree(g.V, g.E, off, dev_u32(bad), None, noff, nsrc, None, o2n)
    boff = g.offsets.copy()
    boff[5] = boff[6] + 1
    with pytest.raises(wedge.WedgeError, match="non-decreasing"):
        wedge.wedge_csc_relabel_by_degree(g.V, g.E, dev_u32(boff), src, None, noff, nsrc, None, o2n)
    with pytest.raises(wedge.WedgeError, match="both"):
        wedge.wedge_csc_relabel_by_degree(g.V, g.E, off, src, dev_u32(g.w), noff, nsrc, None, o2n)
    with pytest.raises(wedge.WedgeError, match="device memory"):
        wedge.wedge_csc_relabel_by_degree(g.V, g.E, g.offsets, src, None, noff, nsrc, None, o2n)
    with pytest.raises(wedge.WedgeError):
        wedge.wedge_permute_rows(g.V, 1, o2n, nsrc, nsrc)
