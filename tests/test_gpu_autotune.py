"""The autotuner's settings change the schedule, never the result: every
setting it times gives bit-identical output, and the chosen one is the
fastest it measured."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _gpu import graph
from paper_1903_07754_gb300 import autotune, wedge

pytestmark = pytest.mark.gpu


def test_settings_are_bit_exact_and_best_is_fastest():
    g = gg.rmat(15, 16)
    G = graph(g, with_weights=False)
    try:
        grid = {"k": (0, 2), "tau_bp": (100, 2000), "dense_loader": (0, 1), "blocks_per_sm": (0, 2)}
        best, table = autotune.tune(G.handle, "bfs", g.V, 0, grid=grid, reps=1)
        assert best["ms"] == min(r["ms"] for r in table) and len(table) == 16
        want = oracle.bfs_push(g, 0)
        out = torch.empty(g.V, dtype=torch.int32, device="cuda")
        for r in table:
            wedge.wedge_graph_set_tuning(G.handle, r["dense_loader"], r["blocks_per_sm"])
            wedge.wedge_run_bfs(G.handle, 0, out, autotune.opts_for("bfs", r))
            np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want)
        # several roots: settings ranked by their total time over the roots
        mbest, mtable = autotune.tune(G.handle, "bfs", g.V, [0, 7, 123], grid={"k": (0, 2), "tau_bp": (100,)},
                                      reps=1)
        assert len(mtable) == 2 and mbest["ms"] == min(r["ms"] for r in mtable)
        roots = gg.roots(g, 16, seed=8)
        bbest, btable = autotune.tune(G.handle, "bfs_batch", g.V, roots=roots, nqueries=16,
                                      grid={"k": (0, 3), "tau_bp": (100, 5000), "blocks_per_sm": (0, 1)}, reps=1)
        lv = torch.empty(g.V * 16, dtype=torch.int32, device="cuda")
        for r in btable:
            wedge.wedge_graph_set_tuning(G.handle, 0, r["blocks_per_sm"])
            wedge.wedge_run_bfs_batch(G.handle, roots, None, 16, lv, autotune.opts_for("bfs_batch", r))
            got = lv.cpu().numpy().view(np.uint32).reshape(g.V, 16)
            for q in (0, 7, 15):
                np.testing.assert_array_equal(got[:, q], oracle.bfs_push(g, int(roots[q])))
    finally:
        G.close()
