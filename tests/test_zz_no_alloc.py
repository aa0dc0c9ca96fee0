"""The allocation-free transformation entry point.

It serves callers that cannot call cudaMalloc (a framework that owns the
device memory pool, latency-critical loops, fixed device footprints).  Its
result must equal wedge_frontier_transform's on the same inputs, on two calls
in a row (the second call reuses the library's fixed scratch array left by
the first), and the Wedge Frontier's definition computed by the oracle.  This file sorts last so a run that stops at its first failure
has already run every other test."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from paper_1903_07754_gb300 import wedge


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _bitmap(V, mask):
    bits = np.zeros(((V + 31) // 32) * 32, dtype=np.uint64)
    bits[:V] = mask
    return (bits.reshape(-1, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


@pytest.mark.gpu
def test_noalloc_transform_matches_transform_twice():
    g = gg.rmat(15, 16)
    G = wedge.Graph.from_csc(g, with_weights=False)
    try:
        info = G.info
        eo = torch.empty(g.V + 1, dtype=torch.int32, device="cuda")
        ei = torch.empty(max(info["eidx_len"], 1), dtype=torch.int32, device="cuda")
        wedge.wedge_graph_copy_edge_index(G.handle, eo, ei)
        nc = info["nchunks"]
        for frac, seed, k in ((0.3, 11, 0), (0.01, 12, 2)):
            r = np.array([gg.rand(seed, i) for i in range(g.V)], dtype=np.uint64)
            mask = (r % np.uint64(1000)) < np.uint64(int(frac * 1000))
            mask[0] = True
            bm = _dev(_bitmap(g.V, mask))
            cap = (nc + (1 << k) - 1) >> k
            want_list = torch.empty(cap, dtype=torch.int32, device="cuda")
            want_n = torch.zeros(1, dtype=torch.int32, device="cuda")
            wedge.wedge_frontier_transform(G.handle, bm, k, want_list, want_n)
            got_list = torch.empty(cap, dtype=torch.int32, device="cuda")
            got_n = torch.full((1,), 7, dtype=torch.int32, device="cuda")  # the call resets the count
            wedge.wedge_frontier_transform_noalloc(g.V, g.E, eo, ei, bm, k, got_list, got_n)
            n, m = int(_host(want_n)[0]), int(_host(got_n)[0])
            assert m == n and n > 0
            np.testing.assert_array_equal(np.sort(_host(got_list)[:m]), np.sort(_host(want_list)[:n]))
            np.testing.assert_array_equal(np.sort(_host(got_list)[:m]).astype(np.uint64),
                                          oracle.wedge_groups_scan(g, mask, 32 << k))
    finally:
        G.close()


def test_noalloc_rejects_graphs_beyond_its_scratch():
    wedge.load()
    one = np.zeros(4, dtype=np.uint32)
    with pytest.raises(wedge.WedgeError) as e:
        # ceil(E/32) = 2^26 + 1 chunk entries > 2^25 at k = 0: rejected before any device work
        wedge.wedge_frontier_transform_noalloc(1, (1 << 31) + 32, one, one, one, 0, one, one, stream=0)
    assert e.value.status == 1
    assert "fixed scratch" in wedge.wedge_last_error()
