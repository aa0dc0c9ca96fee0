"""Trains the learned switch's cost model on the GPU and writes
`cost_model.npy` (and `cost_model.json`, a summary) next to this file.

Training mix: R-MAT scales 18, 20, 22 and 24 (edge factor 16) with a in
{0.45, 0.57, 0.70} (b = c = (1-a)*0.19/0.43, d the rest), and rewired grids
(1024^2 and 2048^2, p = 0.01), BFS and SSSP from seeded roots and CC on the
symmetrised graph, every candidate timed at every iteration (up to 128 per
run).  Held out: R-MAT scale 21, a = 0.57, seed 99.  Also learns the band of
fullness / E outside which the traces' fastest candidate never varied (the
decision skips inference there).

    python -m paper_1903_07754_gb300.train_cost_model [--quick]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
from paper_1903_07754_gb300 import costmodel, wedge  # noqa: E402


def _graph_traces(g, sym, seed, max_iters=128):
    G = wedge.Graph.from_csc(g)
    S = wedge.Graph.from_csc(sym, with_weights=False)
    try:
        roots = gg.roots(g, 2, seed=seed)
        tr = costmodel.collect(G.handle, "bfs", roots, wedge.wedge_default_opts("bfs"), max_iters)
        tr += costmodel.collect(G.handle, "sssp", roots[:1], wedge.wedge_default_opts("sssp"), max_iters)
        tr += costmodel.collect(S.handle, "cc", [0], wedge.wedge_default_opts("cc"), max_iters)
    finally:
        G.close()
        S.close()
    return tr


def rmat_case(scale, a, seed):
    b = (1 - a) * 0.19 / 0.43
    g = gg.rmat(scale, 16, a=a, b=b, c=b, seed=seed).with_weights(255)
    return g, gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))


def grid_case(n, p, seed):
    g = gg.grid(n, p, seed=seed).with_weights(1000)
    return g, g


def main():
    quick = "--quick" in sys.argv
    wedge.load()
    scales = (16, 17) if quick else (18, 20, 22, 24)
    t0 = time.time()
    train = []
    for i, scale in enumerate(scales):
        for j, a in enumerate((0.45, 0.57, 0.70)):
            seed = 100 + 10 * i + j
            train += _graph_traces(*rmat_case(scale, a, seed), seed)
    for n in ((256,) if quick else (1024, 2048)):
        train += _graph_traces(*grid_case(n, 0.01, 4), 7)
    held = _graph_traces(*rmat_case(17 if quick else 21, 0.57, 99), 99)
    X, T = costmodel.dataset(train)
    params, loss = costmodel.train(X, T, steps=3000, lr=3e-3, seed=0)
    # the band ignores the 2% most extreme iterations at each end (single
    # timings of tiny frontiers are noisy)
    band = costmodel.learn_band(train, quantile=0.02)
    learned, threshold, best = costmodel.evaluate(params, held, band)
    learned_tr, threshold_tr, best_tr = costmodel.evaluate(params, train, band)
    costmodel.save(params)
    summary = {"rows": int(len(T)), "iterations": int(sum(len(m) for _, m, _ in train)), "train_loss": loss,
               "band": list(band),
               "held_out": {"graph": "rmat-s%d-a0.57-seed99" % (17 if quick else 21), "regret_learned_ms": learned,
                            "regret_threshold_ms": threshold, "best_total_ms": best},
               "train": {"regret_learned_ms": learned_tr, "regret_threshold_ms": threshold_tr,
                         "best_total_ms": best_tr},
               "seconds": time.time() - t0}
    with open(os.path.join(os.path.dirname(costmodel.DEFAULT_MODEL), "cost_model.json"), "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
