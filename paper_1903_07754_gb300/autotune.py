"""Autotuner for the pull schedule (not in the paper).

For one graph and application it times a grid of settings -- Wedge Frontier
precision k (entries of 32*2^k edges; k = -1, -2: 16 and 8 edges), fullness threshold tau, dense loader
(direct streaming loads or bulk-copy staging), pull blocks per SM and the
edge index the transformation reads (plain or compressed) -- with CUDA
events, and returns the fastest.  Every setting computes the same
result (the schedule never changes the fixed point; BFS is level-exact), so
tuning is safe; `tests/test_gpu_autotune.py` checks that the chosen and
rejected settings agree bit for bit.  Results can be cached in a JSON file
keyed by graph size and application.
"""
from __future__ import annotations

import itertools
import json
import os

from . import wedge

DEFAULT_GRID = {
    "bfs": {"k": (-2, -1, 0, 1, 2, 3), "tau_bp": (50, 100, 500, 2000), "dense_loader": (0,), "blocks_per_sm": (0,),
            "edge_index": (0,)},
    "cc": {"k": (-2, -1, 0, 1, 2), "tau_bp": (500, 2000, 5000), "dense_loader": (0, 1), "blocks_per_sm": (0,),
           "edge_index": (0,)},
    "sssp": {"k": (-2, -1, 0, 1, 2), "tau_bp": (100, 500, 2000), "dense_loader": (0, 1), "blocks_per_sm": (0,),
             "edge_index": (0,)},
    "bfs_batch": {"k": (0, 1, 2, 3, 4), "tau_bp": (100, 500, 2000, 5000), "dense_loader": (0,),
                  "blocks_per_sm": (0,), "edge_index": (0,)},
}


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(handle, app, V, root=0, roots=None, nqueries=64, grid=None, reps=3):
    """Times every setting of `grid` for `app` ('bfs', 'cc', 'sssp' or
    'bfs_batch') on graph `handle`; returns (best setting, table).  `root`
    may be a list: BFS and SSSP settings are then ranked by their total time
    over those roots (a single root can favour a setting that suits only
    it); CC has no root; `roots` are the batched queries' roots."""
    import torch
    grid = dict(DEFAULT_GRID[app], **(grid or {}))
    out = torch.empty(V * (nqueries if app == "bfs_batch" else 1), dtype=torch.int32, device="cuda")
    base_app = "bfs" if app == "bfs_batch" else app
    tune_roots = [int(r) for r in root] if hasattr(root, "__len__") else [int(root)]
    before = wedge.wedge_graph_get_tuning(handle)
    table = []
    try:
        for k, tau, loader, bps, ei in itertools.product(grid["k"], grid["tau_bp"], grid["dense_loader"],
                                                         grid["blocks_per_sm"], grid["edge_index"]):
            wedge.wedge_graph_set_tuning(handle, loader, bps, ei)
            o = wedge.wedge_default_opts(base_app)
            o.log2_coarsen, o.tau_bp = k & 0xFFFFFFFF, tau
            if app == "bfs":
                fns = [lambda r=r: wedge.wedge_run_bfs(handle, r, out, o, False) for r in tune_roots]
            elif app == "cc":
                fns = [lambda: wedge.wedge_run_cc(handle, out, o, False)]
            elif app == "sssp":
                fns = [lambda r=r: wedge.wedge_run_sssp(handle, r, out, o, False) for r in tune_roots]
            else:
                fns = [lambda: wedge.wedge_run_bfs_batch(handle, roots, None, nqueries, out, o, False)]
            table.append({"k": k, "tau_bp": tau, "dense_loader": loader, "blocks_per_sm": bps, "edge_index": ei,
                          "ms": sum(_time(fn, reps) for fn in fns)})
    finally:
        wedge.wedge_graph_set_tuning(handle, before["dense_loader"], before["blocks_per_sm"], before["edge_index"])
    best = min(table, key=lambda r: r["ms"])
    return best, table


def apply(handle, best):
    """Installs the best setting's tuning on the graph and returns matching
    options for its application."""
    wedge.wedge_graph_set_tuning(handle, best["dense_loader"], best["blocks_per_sm"], best.get("edge_index", 0))
    return best


def opts_for(app, best):
    o = wedge.wedge_default_opts("bfs" if app == "bfs_batch" else app)
    o.log2_coarsen, o.tau_bp = best["k"] & 0xFFFFFFFF, best["tau_bp"]
    return o


def cached(path, key, compute):
    """JSON cache: returns data[key], computing and storing it if absent."""
    data = {}
    if path and os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    if key not in data:
        data[key] = compute()
        if path:
            with open(path, "w") as f:
                json.dump(data, f, indent=1)
    return data[key]
