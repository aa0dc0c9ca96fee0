"""Benchmark of the Wedge hot path on one GB300 (or N replicas).

One step = BFS (root 0), CC (HCC on the symmetrised graph), SSSP (root 0,
weights in [1,255]) and PageRank (20 iterations, d = 0.85) on R-MAT scale 22,
edge factor 16 (a=0.57, b=c=0.19, seeded, self-loops and duplicates removed),
uint32 CSC resident in HBM, through the C ABI with the precision and
fullness threshold the project's autotuner picks per application (the
paper's settings, 1% / 20% and one 32-edge chunk per Wedge bit, are timed
beside them).

`value` is whole-job GTEPS over the step: traversed edges of every run
(BFS, SSSP: sum of out-degrees of reached vertices; CC: |E_sym|; PR: 20*|E|)
divided by the step time.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SCALE, EF = 22, 16
PR_ITERS, DAMPING = 20, 0.85
WMAX = 255
METRIC = "GTEPS (BFS+CC+SSSP+PR) on R-MAT s22 ef16, Wedge pull vs dense pull, % of HBM roofline"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def make_inputs(scale=SCALE):
    import graphgen as gg
    g = gg.rmat(scale, EF).with_weights(WMAX)
    s = gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))
    return g, s


def credited_edges(outdeg, reached_mask):
    return int(outdeg[reached_mask].sum())


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            # start timing only once the sampler reports, so samples cover the timed region
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, x in enumerate(r[2]) if x.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal

# settings the autotuner tries for the step (direct loads, all blocks per SM).
# Entries of whole chunks only: 8- and 16-edge entries make the resident runs
# 1-3% faster at R-MAT s22 (per_app.precision_ms), but their edge index
# costs about as much to build as the chunk index, once per graph, which
# the end-to-end step (two graph creations) would pay every step.
STEP_TUNE_GRID = {
    "bfs": {"k": (0, 1, 2, 3), "tau_bp": (100, 500, 2000, 5000), "dense_loader": (0,), "blocks_per_sm": (0,)},
    "cc": {"k": (0, 1, 2), "tau_bp": (500, 2000, 5000), "dense_loader": (0,), "blocks_per_sm": (0,)},
    "sssp": {"k": (0, 1, 2), "tau_bp": (100, 500, 2000), "dense_loader": (0,), "blocks_per_sm": (0,)},
}


# fullness thresholds (basis points of |E|) tried for the push/pull hybrid
HYBRID_TAUS = (100, 500, 2000, 5000)


def tune_step(wedge, G, S, g):
    """Wedge Frontier precision and fullness threshold per application,
    picked by the project's autotuner on the step's graphs: the setting with
    the least total time over three roots other than the measured one (CC
    has no root).  The paper's own settings are timed in per_app as well."""
    import graphgen as gg
    from paper_1903_07754_gb300 import autotune
    roots = [int(r) for r in gg.roots(g, 3, seed=7)]
    tuned = {}
    for app, H in (("bfs", G), ("cc", S), ("sssp", G)):
        best, _ = autotune.tune(H.handle, app, g.V, root=roots, grid=STEP_TUNE_GRID[app], reps=3)
        tuned[app] = {"k": best["k"], "tau_bp": best["tau_bp"]}
    return tuned


def step_opts(wedge, app, tuned):
    o = wedge.wedge_default_opts(app)
    o.log2_coarsen, o.tau_bp = tuned[app]["k"] & 0xFFFFFFFF, tuned[app]["tau_bp"]
    return o


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------
# Reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
REF_BUDGET_S = 90.0   # timed seconds of the reference arm at most


def reference_units(g, s, od):
    """The reference arm's bounded samples of the step, in rotation: the
    oracle's full-size BFS (push), CC (union-find), SSSP (Dijkstra) and two
    PageRank iterations (FP64 pull); each returns the edges it is credited
    with, counted as in our arm."""
    import oracle

    def bfs():
        return credited_edges(od, oracle.bfs_push(g, 0) != 0xFFFFFFFF)

    def cc():
        oracle.cc_union_find(s)
        return s.E

    def sssp():
        return credited_edges(od, oracle.sssp_dijkstra(g, 0) != 0xFFFFFFFF)

    def pr2():
        oracle.pr_pull(g, DAMPING, 2)
        return 2 * g.E
    return [("bfs", bfs), ("cc", cc), ("sssp", sssp), ("pr2", pr2)]


def reduce_max(value, world, device):
    """Max over ranks (the slowest replica sets the job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The oracle timed on the host cores, rank 0 only (other ranks exit at
    once).  A step is one bounded sample (reference_units, in rotation);
    steps stop early once REF_BUDGET_S timed seconds are spent, so the run
    ends within a few minutes for any --steps."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    g, s = make_inputs(args.scale)
    od = oracle.outdeg(g)
    units = reference_units(g, s, od)
    for i in range(min(max(args.warmup, 0), 1)):
        units[i % len(units)][1]()
    t_total, edges, done = 0.0, 0, 0
    while done < args.steps and (t_total < REF_BUDGET_S or done < len(units)):
        t0 = time.perf_counter()
        edges += units[done % len(units)][1]()
        t_total += time.perf_counter() - t0
        done += 1
    value = edges / t_total / 1e9
    sample = (f"oracle (single-threaded C) on the full-size graphs, one unit per step in rotation: push BFS, "
              f"union-find CC, Dijkstra SSSP, 2 FP64 PageRank iterations; {done} of {args.steps} steps "
              f"({t_total:.1f} s timed, budget {REF_BUDGET_S:.0f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": done, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * t_total / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f64",
            "data": "synthetic", "config": {"workload": f"rmat-s{args.scale}-ef{EF}: bfs+cc(sym)+sssp+pr{PR_ITERS}"},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


# --------------------------------------------------------------------------
# Our arm
# --------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--ref-pr-iters", type=int, default=PR_ITERS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    choices=["cc-dense", "pr", "pr-relabel", "step", "frontier-traced", "xform"],
                    help="run only one small case for a profiler (no JSON line)")
    ap.add_argument("--config", default="s22", choices=["s22", "learned-s24", "batch-s26", "grid", "studies"],
                    help="s22: the benchmark line (R-MAT s22, four apps); the others print one line each "
                         "for the learned switch (R-MAT s24), batched traversal (R-MAT s26, uneven "
                         "batch), the rewired grid and the paper's studies (time split, per-iteration "
                         "profiles, threshold and precision sweeps)")
    args = ap.parse_args()

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import oracle
    from paper_1903_07754_gb300 import wedge

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    from paper_1903_07754_gb300 import build as wbuild
    wbuild.build()
    wedge.load()
    if args.config != "s22":
        # clocks sampled over the whole configuration (its timed regions and
        # the input generation between them)
        with ClockSampler(local) as clk:
            line = {"learned-s24": bench_learned, "batch-s26": bench_batch, "grid": bench_grid,
                    "studies": bench_studies}[args.config](
                args, wedge, torch, dev, world)
        line["clocks"] = clk.summary()
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    g, s = make_inputs(args.scale)
    od = oracle.outdeg(g)
    G = wedge.Graph.from_csc(g)
    S = wedge.Graph.from_csc(s, with_weights=False)
    if args.profile_case:
        if args.profile_case == "cc-dense":
            print(json.dumps(roofline_dense_pull(wedge, torch, G, S, g, s, stream, dev)))
        elif args.profile_case == "step":
            # the step's kernels with the profiler on only around the steps
            # (ncu --profile-from-start off); BFS, CC and SSSP run their
            # iterations through the host-polled loop (traced runs: the same
            # kernels and launch shapes) so that every launch is visible
            tuned = tune_step(wedge, G, S, g)
            o = [step_opts(wedge, a, tuned) for a in ("bfs", "cc", "sssp")]
            for x in o:
                x.trace = 1
            out = torch.empty(g.V, dtype=torch.int32, device=dev)
            r = torch.empty(g.V, dtype=torch.float32, device=dev)

            def one():
                wedge.wedge_run_bfs(G.handle, 0, out, o[0], False)
                wedge.wedge_run_cc(S.handle, out, o[1], False)
                wedge.wedge_run_sssp(G.handle, 0, out, o[2], False)
                wedge.wedge_run_pr(G.handle, r, PR_ITERS, DAMPING, None, False)
            one()
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStart()
            for _ in range(args.steps):
                one()
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()
        elif args.profile_case == "xform":
            print(json.dumps(transform_case(wedge, torch, G, g, od, stream, dev)))
        elif args.profile_case in ("pr", "pr-relabel"):
            H = G
            if args.profile_case == "pr-relabel":  # the same pulls on the degree-relabelled copy
                arr = [torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev) for a in (g.offsets, g.src)]
                noff = torch.empty(g.V + 1, dtype=torch.int32, device=dev)
                nsrc = torch.empty(g.E, dtype=torch.int32, device=dev)
                o2n = torch.empty(g.V, dtype=torch.int32, device=dev)
                wedge.wedge_csc_relabel_by_degree(g.V, g.E, arr[0], arr[1], None, noff, nsrc, None, o2n)
                H = wedge.Graph(wedge.wedge_graph_create(g.V, g.E, noff, nsrc), keep=[noff, nsrc])
            r = torch.empty(g.V, dtype=torch.float32, device=dev)
            for _ in range(2):
                wedge.wedge_run_pr(H.handle, r, 3, DAMPING, None, False)
            torch.cuda.synchronize()
            if H is not G:
                H.close()
        else:
            # the step's frontier runs through the host-polled loop (traced
            # runs), so that a profiler sees every kernel launch
            out = torch.empty(g.V, dtype=torch.int32, device=dev)
            for a, h in (("bfs", G), ("cc", S), ("sssp", G)):
                o = wedge.wedge_default_opts(a)
                o.trace = 1
                fn = {"bfs": lambda: wedge.wedge_run_bfs(h.handle, 0, out, o, False),
                      "cc": lambda: wedge.wedge_run_cc(h.handle, out, o, False),
                      "sssp": lambda: wedge.wedge_run_sssp(h.handle, 0, out, o, False)}[a]
                fn()
            torch.cuda.synchronize()
        G.close()
        S.close()
        return
    V = g.V
    lvl = torch.empty(V, dtype=torch.int32, device=dev)
    lab = torch.empty(V, dtype=torch.int32, device=dev)
    dist_ = torch.empty(V, dtype=torch.int32, device=dev)
    rank_t = torch.empty(V, dtype=torch.float32, device=dev)
    tuned = tune_step(wedge, G, S, g)
    o_bfs, o_cc, o_sssp = (step_opts(wedge, a, tuned) for a in ("bfs", "cc", "sssp"))

    def step(want_stats=False):
        sb = wedge.wedge_run_bfs(G.handle, 0, lvl, o_bfs, want_stats)
        sc = wedge.wedge_run_cc(S.handle, lab, o_cc, want_stats)
        ss = wedge.wedge_run_sssp(G.handle, 0, dist_, o_sssp, want_stats)
        sp = wedge.wedge_run_pr(G.handle, rank_t, PR_ITERS, DAMPING, None, want_stats)
        return sb, sc, ss, sp

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    # credited edges are fixed by the result (checked once)
    step()
    torch.cuda.synchronize()
    lv = lvl.cpu().numpy().view(np.uint32)
    dv = dist_.cpu().numpy().view(np.uint32)
    edges = {"bfs": credited_edges(od, lv != 0xFFFFFFFF), "cc": s.E,
             "sssp": credited_edges(od, dv != 0xFFFFFFFF), "pr": PR_ITERS * g.E}
    step_edges = sum(edges.values())

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    launches0 = wedge.wedge_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
    launches = wedge.wedge_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    ms = reduce_max(ms, world, dev)
    ms_per_step = ms / args.steps
    value = world * step_edges * args.steps / (ms / 1e3) / 1e9
    # end to end through host buffers, before the studies below fill the
    # device's memory pools
    e2e = e2e_measure(wedge, torch, g, s, od, edges, args, dev, (o_bfs, o_cc, o_sssp)) \
        if rank == 0 and not args.no_e2e else None

    # per-app ms/run (median of 10 runs after 2 warm-ups, CUDA events per
    # run) in every mode: Wedge with the fixed threshold (default options),
    # dense pull every iteration, Wedge Frontier every iteration, learned
    per_app = {}
    dense = {a: wedge.wedge_default_opts(a) for a in ("bfs", "cc", "sssp")}
    sparse = {a: wedge.wedge_default_opts(a) for a in ("bfs", "cc", "sssp")}
    for a in dense.values():
        a.switch_mode = wedge.SWITCH_ALWAYS_DENSE
    for a in sparse.values():
        a.switch_mode = wedge.SWITCH_ALWAYS_SPARSE

    def time_fn(fn, reps=10):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    runs = {
        "bfs": (lambda o: wedge.wedge_run_bfs(G.handle, 0, lvl, o, False), o_bfs, dense["bfs"]),
        "cc": (lambda o: wedge.wedge_run_cc(S.handle, lab, o, False), o_cc, dense["cc"]),
        "sssp": (lambda o: wedge.wedge_run_sssp(G.handle, 0, dist_, o, False), o_sssp, dense["sssp"]),
    }
    stat_fn = {"bfs": lambda o: wedge.wedge_run_bfs(G.handle, 0, lvl, o),
               "cc": lambda o: wedge.wedge_run_cc(S.handle, lab, o),
               "sssp": lambda o: wedge.wedge_run_sssp(G.handle, 0, dist_, o)}
    for name, (fn, ow, odn) in runs.items():
        t_w = time_fn(lambda: fn(ow))
        t_d = time_fn(lambda: fn(odn))
        t_s = time_fn(lambda: fn(sparse[name]))
        t_p = time_fn(lambda: fn(wedge.wedge_default_opts(name)))
        sd = stat_fn[name](odn)
        # the Wedge Frontier's precision at the tuned threshold: entries of
        # 8, 16 and 32 edges (k = -2, -1, 0; Section 3.4 "Frontier Precision")
        by_k = {}
        for k in (-2, -1, 0):
            ok = step_opts(wedge, name, tuned)
            ok.log2_coarsen = k & 0xFFFFFFFF
            by_k[f"k{k}"] = time_fn(lambda: fn(ok))
        per_app[name] = {"ms": t_w, "gteps": edges[name] / (t_w / 1e3) / 1e9, "tuned": tuned[name],
                         "precision_ms": by_k,
                         "paper_settings_ms": t_p, "dense_pull_ms": t_d,
                         "speedup_vs_dense_pull": t_d / t_w, "always_sparse_ms": t_s,
                         "speedup_vs_always_sparse": t_s / t_w,
                         "dense_pull_edges_per_s": sd.edges_pulled / (t_d / 1e3)}
    # learned switch (cost model trained by paper_1903_07754_gb300.train_cost_model)
    from paper_1903_07754_gb300 import costmodel
    if os.path.exists(costmodel.DEFAULT_MODEL):
        params = costmodel.load_params()
        band = costmodel.load_band()
        for H in (G, S):
            wedge.wedge_set_cost_model(H.handle, params)
            wedge.wedge_set_learned_band(H.handle, *band)
        for name, (fn, ow, _) in runs.items():
            ol = wedge.wedge_default_opts(name)
            ol.switch_mode = wedge.SWITCH_LEARNED
            t_l = time_fn(lambda: fn(ol))
            per_app[name]["learned_ms"] = t_l
            per_app[name]["speedup_learned_vs_threshold"] = per_app[name]["ms"] / t_l
            per_app[name]["speedup_learned_vs_paper_settings"] = per_app[name]["paper_settings_ms"] / t_l
            per_app[name]["speedup_learned_vs_dense_pull"] = per_app[name]["dense_pull_ms"] / t_l
        for H in (G, S):
            wedge.wedge_set_cost_model(H.handle, None)
            wedge.wedge_set_learned_band(H.handle, *costmodel.NO_BAND)
    # the push/pull hybrid (the comparison engine: sparse iterations push
    # over the frontier's out-edges, dense ones pull), its threshold tuned
    # on the tuning roots like Wedge's settings, timed on the measured root
    import graphgen as gg
    troots = [int(r) for r in gg.roots(g, 3, seed=7)]

    def run_app(name, o, root):
        if name == "bfs":
            return wedge.wedge_run_bfs(G.handle, root, lvl, o, False)
        if name == "cc":
            return wedge.wedge_run_cc(S.handle, lab, o, False)
        return wedge.wedge_run_sssp(G.handle, root, dist_, o, False)

    def hybrid_opts(name, tau, always_push=False):
        o = wedge.wedge_default_opts(name)
        o.sparse_push = 1
        o.tau_bp = tau
        if always_push:
            o.switch_mode = wedge.SWITCH_ALWAYS_SPARSE
        return o

    for name in runs:
        t_best, tau_best = None, None
        for tau in HYBRID_TAUS:
            oh = hybrid_opts(name, tau)
            t = sum(time_fn(lambda: run_app(name, oh, r), reps=3) for r in (troots[:1] if name == "cc" else troots))
            if t_best is None or t < t_best:
                t_best, tau_best = t, tau
        by_tau = {}
        for tau in HYBRID_TAUS:
            oh = hybrid_opts(name, tau)
            by_tau[str(tau)] = time_fn(lambda: run_app(name, oh, 0), reps=5)
        oh = hybrid_opts(name, tau_best)
        t_h = time_fn(lambda: run_app(name, oh, 0))
        op = hybrid_opts(name, tau_best, always_push=True)
        t_pp = time_fn(lambda: run_app(name, op, 0))
        t_best = min(by_tau.values())
        per_app[name].update({"push_pull_hybrid_ms": t_h, "push_pull_hybrid_tau_bp": tau_best,
                              "speedup_vs_push_pull_hybrid": t_h / per_app[name]["ms"],
                              "push_pull_hybrid_ms_by_tau_bp": by_tau,
                              "speedup_vs_best_push_pull_hybrid": t_best / per_app[name]["ms"],
                              "push_every_iteration_ms": t_pp})
    t_pr = time_fn(lambda: wedge.wedge_run_pr(G.handle, rank_t, PR_ITERS, DAMPING, None, False))
    per_app["pr"] = {"ms": t_pr, "gteps": edges["pr"] / (t_pr / 1e3) / 1e9}
    st = step(want_stats=True)
    for name, sx in zip(("bfs", "cc", "sssp", "pr"), st):
        per_app[name]["iters"] = sx.iters
        per_app[name]["sparse_iters"] = sx.sparse_iters

    # graph + edge-index build (setup, not in the step): device-resident CSC
    build_ms = {}
    for name, gx, wx in (("rmat", g, True), ("sym", s, False)):
        dev_arr = [torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
                   for a in ((gx.offsets, gx.src, gx.w) if wx else (gx.offsets, gx.src))]
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = wedge.wedge_graph_create(gx.V, gx.E, *dev_arr)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
            wedge.wedge_graph_destroy(h)
        build_ms[name] = float(np.median(ts))
        del dev_arr

    # roofline of the dominant kernel, PageRank's dense pull (20 launches per
    # step), with CUDA events around single launches through its entry point
    # on the same stream; and of the first dense CC pull
    roof = roofline_pr_pull(wedge, torch, G, g, stream, dev, clk.summary())
    roof["share_of_step"] = PR_ITERS * roof["ms"] / ms_per_step
    roof_cc = roofline_dense_pull(wedge, torch, G, S, g, s, stream, dev)
    balance = transform_balance(wedge, torch, G, g, stream, dev)
    zindex = compressed_index(wedge, torch, G, g, od, stream, dev, o_sssp)
    locality = locality_study(wedge, torch, g, s, (o_bfs, o_cc, o_sssp), stream, dev, time_fn, ms_per_step)

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
            "config": {"workload": f"rmat-s{args.scale}-ef{EF}: bfs+cc(sym)+sssp+pr{PR_ITERS}",
                       "V": V, "E": g.E, "E_sym": s.E, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (CSC src alone is %d MB)" % (4 * g.E >> 20),
                       "wedge_settings": "autotuned (k, tau) per app: " + json.dumps(tuned)},
            "per_app": per_app, "graph_build_ms": build_ms, "roofline": roof, "roofline_cc_dense_pull": roof_cc,
            "transform_balance": balance, "compressed_edge_index": zindex, "locality_relabel": locality,
            "gpu_launches": int(launches),
            "clocks": clk.summary()}
    if e2e is not None:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, s, od)
    G.close()
    S.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def locality_study(wedge, torch, g, s, opts, stream, dev, time_fn, step_ms):
    """The benchmark step on degree-relabelled copies of its two graphs
    (wedge_csc_relabel_by_degree: new ids by descending out-degree, so the
    most gathered values share cache lines; not in the paper), with the
    same tuned options: the relabelling's device time, each application's
    time with and without bringing its result back to the original ids,
    the whole step, and the PageRank pull's gather rate."""
    V = g.V
    o_bfs, o_cc, o_sssp = opts
    src_d = {}
    for name, gx, wx in (("rmat", g, True), ("sym", s, False)):
        arr = [torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
               for a in ((gx.offsets, gx.src, gx.w) if wx else (gx.offsets, gx.src))]
        out = {"off": torch.empty(gx.V + 1, dtype=torch.int32, device=dev),
               "src": torch.empty(gx.E, dtype=torch.int32, device=dev),
               "w": torch.empty(gx.E, dtype=torch.int32, device=dev) if wx else None,
               "o2n": torch.empty(gx.V, dtype=torch.int32, device=dev),
               "n2o": torch.empty(gx.V, dtype=torch.int32, device=dev)}

        def relabel():
            wedge.wedge_csc_relabel_by_degree(gx.V, gx.E, arr[0], arr[1], arr[2] if wx else None, out["off"],
                                              out["src"], out["w"], out["o2n"], out["n2o"], stream=stream)
        out["t"] = _time_launch(torch, stream, relabel, reps=3, warm=1)
        src_d[name] = out
        del arr
    R, Sd = src_d["rmat"], src_d["sym"]
    G = wedge.Graph(wedge.wedge_graph_create(V, g.E, R["off"], R["src"], R["w"]), keep=[R["off"], R["src"], R["w"]])
    S = wedge.Graph(wedge.wedge_graph_create(s.V, s.E, Sd["off"], Sd["src"]), keep=[Sd["off"], Sd["src"]])
    root = int(R["o2n"][0].item())
    a = torch.empty(V, dtype=torch.int32, device=dev)
    b = torch.empty(V, dtype=torch.int32, device=dev)
    c = torch.empty(V, dtype=torch.int32, device=dev)
    r = torch.empty(V, dtype=torch.float32, device=dev)
    rb = torch.empty(V, dtype=torch.float32, device=dev)
    runs = {"bfs": lambda: wedge.wedge_run_bfs(G.handle, root, a, o_bfs, False),
            "cc": lambda: wedge.wedge_run_cc(S.handle, a, o_cc, False),
            "sssp": lambda: wedge.wedge_run_sssp(G.handle, root, a, o_sssp, False),
            "pr": lambda: wedge.wedge_run_pr(G.handle, r, PR_ITERS, DAMPING, None, False)}
    back = {"bfs": lambda: wedge.wedge_permute_rows(V, 1, R["o2n"], a, b),
            "cc": lambda: wedge.wedge_cc_labels_to_original(s.V, Sd["n2o"], a, c, b),
            "sssp": lambda: wedge.wedge_permute_rows(V, 1, R["o2n"], a, b),
            "pr": lambda: wedge.wedge_permute_rows(V, 1, R["o2n"], r, rb)}
    per_app = {}
    for name in runs:
        t = time_fn(runs[name])
        tb = time_fn(lambda: (runs[name](), back[name]()))
        per_app[name] = {"ms": t, "ms_with_map_back": tb}

    def step():
        for name in ("bfs", "cc", "sssp", "pr"):
            runs[name]()
            back[name]()
    t_step = time_fn(step, reps=20)
    od = torch.from_numpy(g.outdeg().astype(np.float32)).to(dev)
    od_new = torch.empty_like(od)
    wedge.wedge_permute_rows(V, 1, R["n2o"], od, od_new)  # out-degree of new vertex i
    contrib = torch.where(od_new > 0, (1.0 / V) / torch.clamp(od_new, min=1.0), torch.zeros_like(od_new)).contiguous()
    sums = torch.zeros(V, dtype=torch.int64, device=dev)
    t_pull = _time_launch(torch, stream, lambda: wedge.wedge_pr_pull(G.handle, contrib, sums),
                          before=lambda: sums.zero_(), reps=10)
    G.close()
    S.close()
    return {"relabel_ms": {"rmat": R["t"] * 1e3, "sym": Sd["t"] * 1e3}, "per_app": per_app,
            "step_ms_with_map_back": t_step, "speedup_step": step_ms / t_step,
            "pr_pull_ms": t_pull * 1e3, "pr_pull_gathers_gs": g.E / t_pull / 1e9,
            "note": "not in the paper: a locality step before graph creation; the main step runs on the "
                    "graphs as generated"}


def _events(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _base_line(metric, value, unit, ms, steps, world, config, dtype="u32"):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": steps, "warmup": 3,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config}


def bench_learned(args, wedge, torch, dev, world):
    """Learned switch vs fixed threshold vs dense pull: BFS and SSSP on R-MAT
    s24 ef16 (16.8 M vertices), root 0."""
    import graphgen as gg
    import oracle
    from paper_1903_07754_gb300 import costmodel
    g = gg.rmat(24, EF).with_weights(WMAX)
    od = oracle.outdeg(g)
    G = wedge.Graph.from_csc(g)
    out = torch.empty(g.V, dtype=torch.int32, device=dev)
    params = costmodel.load_params()
    res = {}
    total_edges, total_ms = 0, 0.0
    for app in ("bfs", "sssp"):
        run = (lambda o: wedge.wedge_run_bfs(G.handle, 0, out, o, False)) if app == "bfs" else \
            (lambda o: wedge.wedge_run_sssp(G.handle, 0, out, o, False))
        thr = wedge.wedge_default_opts(app)
        dense = wedge.wedge_default_opts(app)
        dense.switch_mode = wedge.SWITCH_ALWAYS_DENSE
        learned = wedge.wedge_default_opts(app)
        learned.switch_mode = wedge.SWITCH_LEARNED
        t_thr = _events(torch, lambda: run(thr), 5)
        t_dense = _events(torch, lambda: run(dense), 5)
        wedge.wedge_set_cost_model(G.handle, params)
        wedge.wedge_set_learned_band(G.handle, *costmodel.load_band())
        t_l = _events(torch, lambda: run(learned), 5)
        wedge.wedge_set_cost_model(G.handle, None)
        wedge.wedge_set_learned_band(G.handle, *costmodel.NO_BAND)
        run(thr)
        torch.cuda.synchronize()
        reached = out.cpu().numpy().view(np.uint32) != 0xFFFFFFFF
        edges = credited_edges(od, reached)
        res[app] = {"learned_ms": t_l, "threshold_ms": t_thr, "dense_pull_ms": t_dense,
                    "speedup_learned_vs_threshold": t_thr / t_l, "speedup_learned_vs_dense_pull": t_dense / t_l,
                    "gteps_learned": edges / (t_l / 1e3) / 1e9}
        total_edges += edges
        total_ms += t_l
    G.close()
    line = _base_line("GTEPS (BFS+SSSP, learned switch) on R-MAT s24 ef16", total_edges / (total_ms / 1e3) / 1e9,
                      "GTEPS", total_ms, 5, world, {"workload": "rmat-s24-ef16: bfs+sssp, learned switch",
                                                    "V": g.V, "E": g.E})
    line["per_app"] = res
    return line


def bench_batch(args, wedge, torch, dev, world):
    """Batched BFS and SSSP: 64 and 1024 roots (seeded, uniform over vertices
    with out-edges) on R-MAT s26 ef16 in waves of 64 queries, and an uneven
    batch of 256 R-MAT graphs of scales 12..20 (block-diagonal, one root
    each)."""
    import graphgen as gg
    from paper_1903_07754_gb300 import autotune
    scale = 26 if args.scale == SCALE else args.scale
    g = gg.rmat(scale, EF).with_weights(WMAX)
    od = g.outdeg()
    G = wedge.Graph.from_csc(g)
    roots = gg.roots(g, 1024, seed=3)
    lv = torch.empty(g.V * 64, dtype=torch.int32, device=dev)
    best, table = autotune.tune(G.handle, "bfs_batch", g.V, roots=roots[:64], nqueries=64,
                                grid={"k": (1, 2, 3), "tau_bp": (500, 2000, 5000)}, reps=1)
    autotune.apply(G.handle, best)
    o = autotune.opts_for("bfs_batch", best)
    res = {"autotuned": {k: best[k] for k in ("k", "tau_bp", "dense_loader", "blocks_per_sm")}}
    wedge.wedge_run_bfs_batch(G.handle, roots[:64], None, 64, lv, o, False)
    od_t = torch.from_numpy(od.astype(np.int64)).to(dev)
    edges64 = _batch_edges(torch, lv, od_t, g.V)
    t64 = _events(torch, lambda: wedge.wedge_run_bfs_batch(G.handle, roots[:64], None, 64, lv, o, False), 3)

    def waves():
        for w in range(16):
            wedge.wedge_run_bfs_batch(G.handle, roots[64 * w:64 * (w + 1)], None, 64, lv, o, False)
    t1024 = _events(torch, waves, 1)
    res["roots64"] = {"ms": t64, "gteps": edges64 / (t64 / 1e3) / 1e9}
    res["roots1024"] = {"ms": t1024, "gteps_est": 16 * edges64 / (t1024 / 1e3) / 1e9,
                        "note": "traversed edges estimated from the first wave"}
    # the same queries with 8-bit levels (a quarter of the output's memory
    # and writes; the call checks that every level fits)
    lv8 = torch.empty(g.V * 64, dtype=torch.uint8, device=dev)
    wedge.wedge_run_bfs_batch_u8(G.handle, roots[:64], None, 64, lv8, o, False)
    wedge.wedge_run_bfs_batch(G.handle, roots[:64], None, 64, lv, o, False)
    same = bool(torch.equal(lv8, torch.where(lv == -1, torch.full_like(lv, 255), lv).to(torch.uint8)))
    t64_8 = _events(torch, lambda: wedge.wedge_run_bfs_batch_u8(G.handle, roots[:64], None, 64, lv8, o, False), 3)

    def waves8():
        for w in range(16):
            wedge.wedge_run_bfs_batch_u8(G.handle, roots[64 * w:64 * (w + 1)], None, 64, lv8, o, False)
    t1024_8 = _events(torch, waves8, 1)
    res["roots64_u8"] = {"ms": t64_8, "gteps": edges64 / (t64_8 / 1e3) / 1e9, "equal_to_u32_levels": same}
    res["roots1024_u8"] = {"ms": t1024_8, "gteps_est": 16 * edges64 / (t1024_8 / 1e3) / 1e9}
    del lv8
    # batched SSSP (weights in [1, 255]) from the same roots
    wedge.wedge_run_sssp_batch(G.handle, roots[:64], None, 64, lv, None, False)
    sedges64 = _batch_edges(torch, lv, od_t, g.V)
    ts64 = _events(torch, lambda: wedge.wedge_run_sssp_batch(G.handle, roots[:64], None, 64, lv, None, False), 3)

    def swaves():
        for w in range(16):
            wedge.wedge_run_sssp_batch(G.handle, roots[64 * w:64 * (w + 1)], None, 64, lv, None, False)
    ts1024 = _events(torch, swaves, 1)
    res["sssp_roots64"] = {"ms": ts64, "gteps": sedges64 / (ts64 / 1e3) / 1e9}
    res["sssp_roots1024"] = {"ms": ts1024, "gteps_est": 16 * sedges64 / (ts1024 / 1e3) / 1e9}
    G.close()
    del lv
    graphs = [gg.rmat(12 + (i % 9), EF, seed=1000 + i).with_weights(WMAX) for i in range(256)]
    big, base = gg.block_diagonal(graphs)
    B = wedge.Graph.from_csc(big)
    lvb = torch.empty(big.V * 64, dtype=torch.int32, device=dev)
    rq = (np.arange(256) % 64).astype(np.uint32)
    tb = _events(torch, lambda: wedge.wedge_run_bfs_batch(B.handle, base.astype(np.uint32), rq, 64, lvb, None, False), 3)
    eb = _batch_edges(torch, lvb, torch.from_numpy(big.outdeg().astype(np.int64)).to(dev), big.V)
    res["uneven256"] = {"ms": tb, "gteps": eb / (tb / 1e3) / 1e9, "V": big.V, "E": big.E}
    tsb = _events(torch, lambda: wedge.wedge_run_sssp_batch(B.handle, base.astype(np.uint32), rq, 64, lvb, None,
                                                            False), 3)
    esb = _batch_edges(torch, lvb, torch.from_numpy(big.outdeg().astype(np.int64)).to(dev), big.V)
    res["sssp_uneven256"] = {"ms": tsb, "gteps": esb / (tsb / 1e3) / 1e9}
    B.close()
    line = _base_line(f"GTEPS (batched BFS, 64 roots) on R-MAT s{scale} ef16", res["roots64"]["gteps"], "GTEPS", t64,
                      3, world, {"workload": f"rmat-s{scale}-ef16: 64/1024-root batched BFS and SSSP + 256-graph uneven batch",
                                 "V": g.V, "E": g.E})
    line["batch"] = res
    return line


def _batch_edges(torch, lv, od_t, V):
    """Sum over queries of the out-degrees of the vertices each reached
    (levels vertex-major, 64 queries), on the device."""
    lvv = lv.view(V, 64)
    return int(sum(int(od_t[lvv[:, q] != -1].sum().item()) for q in range(64)))


def bench_studies(args, wedge, torch, dev, world):
    """The paper's per-application studies, on R-MAT s22 (BFS, SSSP from 0;
    CC on the symmetrised graph): the split of time between pull and
    transformation (Fig. 8), per-iteration dense vs Wedge times with the
    active share of edges (Fig. 9, from the candidate-timing trace), a
    sweep of the fullness threshold including "always transform" (Fig. 10),
    a sweep of the precision (Fig. 11), and for CC and SSSP the iterations
    with in-place updates vs synchronous pulls (Section 5.2's multi-hop
    propagation)."""
    g, s = make_inputs(args.scale)
    G = wedge.Graph.from_csc(g)
    S = wedge.Graph.from_csc(s, with_weights=False)
    out = torch.empty(g.V, dtype=torch.int32, device=dev)
    apps = {"bfs": (G, lambda h, o: wedge.wedge_run_bfs(h, 0, out, o, False)),
            "cc": (S, lambda h, o: wedge.wedge_run_cc(h, out, o, False)),
            "sssp": (G, lambda h, o: wedge.wedge_run_sssp(h, 0, out, o, False))}
    res = {}
    for app, (H, run) in apps.items():
        r = {}
        # Fig. 8: pull vs transformation time (traced run, device timers)
        o = wedge.wedge_default_opts(app)
        o.trace = 1
        run(H.handle, o)
        torch.cuda.synchronize()
        tr = wedge.wedge_get_trace(H.handle)
        r["time_split_ms"] = {"pull": sum(x["t_pull_ns"] for x in tr) / 1e6,
                              "transform": sum(x["t_xform_ns"] for x in tr) / 1e6}
        # Fig. 9: every iteration timed dense and as a Wedge Frontier at the
        # default precision, from the same state
        oc = wedge.wedge_default_opts(app)
        oc.log2_coarsen = 0  # the timed candidates are chunk precisions
        feat, ms, chosen = wedge.wedge_trace_candidates(H.handle, app, 0, oc, 64, 4096)
        kdef = 0
        # feature 3 of the cost model is the fullness over |E|: the active share of edges
        r["per_iteration"] = [{"t": t, "active_edges_pct": 100.0 * float(feat[t, 0, 2]),
                               "dense_ms": float(ms[t, 0]), "wedge_ms": float(ms[t, 1 + kdef]),
                               "threshold_chose": "dense" if chosen[t] == 0 else f"wedge k={int(chosen[t]) - 1}"}
                              for t in range(len(ms))]
        # Fig. 10: fullness threshold (basis points of |E|; 10000 = always transform)
        r["tau_sweep_ms"] = {}
        for tau in (10, 100, 500, 2000, 5000, 10000):
            o = wedge.wedge_default_opts(app)
            o.tau_bp = tau
            r["tau_sweep_ms"][str(tau)] = _events(torch, lambda: run(H.handle, o), 5)
        o = wedge.wedge_default_opts(app)
        o.switch_mode = wedge.SWITCH_ALWAYS_SPARSE
        r["tau_sweep_ms"]["always_transform"] = _events(torch, lambda: run(H.handle, o), 5)
        # Fig. 11: precision, 32 * 2^k edges per Wedge Frontier entry (k = -2,
        # -1: entries of 8 and 16 edges, the paper's finest settings)
        r["precision_sweep_ms"] = {}
        for k in range(-2, 5):
            o = wedge.wedge_default_opts(app)
            o.log2_coarsen = k & 0xFFFFFFFF
            r["precision_sweep_ms"][f"k{k}"] = _events(torch, lambda: run(H.handle, o), 5)
        # multi-hop propagation (Section 5.2): iterations with in-place
        # updates vs every pull reading the previous iteration's values
        if app != "bfs":
            r["multi_hop"] = {}
            for k in (-2, 0, 2, 4):
                row = {}
                for name, sync in (("in_place", 0), ("synchronous", 1)):
                    o = wedge.wedge_default_opts(app)
                    o.log2_coarsen = k & 0xFFFFFFFF
                    o.synchronous = sync
                    st = {"cc": lambda: wedge.wedge_run_cc(H.handle, out, o),
                          "sssp": lambda: wedge.wedge_run_sssp(H.handle, 0, out, o)}[app]()
                    row[f"{name}_iters"] = st.iters
                    row[f"{name}_ms"] = _events(torch, lambda: run(H.handle, o), 3)
                r["multi_hop"][f"k{k}"] = row
        res[app] = r
    G.close()
    S.close()
    t_default = sum(min(v["tau_sweep_ms"].values()) for v in res.values())
    line = _base_line("ms (BFS+CC+SSSP, best threshold) on R-MAT s22 ef16, paper studies", t_default, "ms",
                      t_default, 5, world, {"workload": f"rmat-s{args.scale}-ef{EF}: bfs+cc(sym)+sssp studies"})
    line["higher_is_better"] = False
    line["studies"] = res
    return line


def bench_grid(args, wedge, torch, dev, world):
    """BFS and SSSP (weights in [1,1000]) from vertex 0 on the 4096^2 grid
    with 1% rewiring, and BFS on the plain grid (8190 levels)."""
    import graphgen as gg
    import oracle
    res = {}
    total_e, total_ms = 0, 0.0
    for p_rewire in (0.01, 0.0):
        g = gg.grid(4096, p_rewire).with_weights(1000)
        od = oracle.outdeg(g)
        G = wedge.Graph.from_csc(g)
        out = torch.empty(g.V, dtype=torch.int32, device=dev)
        for app in (("bfs", "sssp") if p_rewire else ("bfs",)):
            run = (lambda o: wedge.wedge_run_bfs(G.handle, 0, out, o, False)) if app == "bfs" else \
                (lambda o: wedge.wedge_run_sssp(G.handle, 0, out, o, False))
            o = wedge.wedge_default_opts(app)
            t = _events(torch, lambda: run(o), 2)
            st = wedge.wedge_run_bfs(G.handle, 0, out, o) if app == "bfs" else wedge.wedge_run_sssp(G.handle, 0, out, o)
            edges = credited_edges(od, out.cpu().numpy().view(np.uint32) != 0xFFFFFFFF)
            res[f"{app}_p{p_rewire:g}"] = {"ms": t, "iters": st.iters, "sparse_iters": st.sparse_iters,
                                           "gteps": edges / (t / 1e3) / 1e9}
            total_e += edges
            total_ms += t
        G.close()
    # multi-hop study (Section 5.2, "Frontier Precision"): with in-place
    # updates, coarser Wedge Frontier entries pull more superfluous edges but
    # carry distances several hops per iteration
    g = gg.grid(4096, 0.01).with_weights(1000)
    G = wedge.Graph.from_csc(g)
    out = torch.empty(g.V, dtype=torch.int32, device=dev)
    study = {}
    for k in (-2, 0, 2, 4, 6):
        o = wedge.wedge_default_opts("sssp")
        o.log2_coarsen = k & 0xFFFFFFFF
        o.switch_mode = wedge.SWITCH_ALWAYS_SPARSE
        t = _events(torch, lambda: wedge.wedge_run_sssp(G.handle, 0, out, o, False), 2)
        st = wedge.wedge_run_sssp(G.handle, 0, out, o)
        study[f"k{k}"] = {"ms": t, "iters": st.iters, "edges_pulled": st.edges_pulled}
        if k in (0, 6):
            # the same pulls reading only the previous iteration's distances
            o.synchronous = 1
            st = wedge.wedge_run_sssp(G.handle, 0, out, o)
            study[f"k{k}"]["synchronous_iters"] = st.iters
    G.close()
    res["sssp_p0.01_always_sparse_by_precision"] = study
    line = _base_line("GTEPS (BFS+SSSP) on the 4096^2 grid", total_e / (total_ms / 1e3) / 1e9, "GTEPS", total_ms, 2,
                      world, {"workload": "grid-4096x4096: p=0.01 bfs+sssp, p=0 bfs"})
    line["per_app"] = res
    return line


# DRAM traffic of one launch (ncu dram__bytes_read.sum + dram__bytes_write.sum),
# that launch's ncu gpu__time_duration in us, and a digest of the device code
# of the captured kernel (KERNEL_FILES): reported only while that code is
# unchanged.  (None, None, None): no capture on the current code yet.
TRAFFIC = {"pr": (314012672, 235.008, "e487f7416430200e"), "cc": (607856896, 505.952, "e487f7416430200e")}
# The sources each captured kernel is built from.
KERNEL_FILES = {"pr": ("pull.cuh", "common.cuh", "tma.cuh", "mlp.cuh"),
                "cc": ("pull.cuh", "common.cuh", "tma.cuh", "mlp.cuh"),
                "xform": ("xform.cuh", "common.cuh")}


def _kernel_digest(key="pr"):
    """Digest of the device code the kernel `key` is built from: comments and
    whitespace are dropped, and so is common.cuh's host part (from the
    host-side graph object on), so that only a change of that device code
    invalidates its counters."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_FILES[key]:
        with open(os.path.join(ROOT, "paper_1903_07754_gb300", "csrc", f)) as fh:
            src = fh.read()
        if f == "common.cuh":
            src = src[:src.index("\nstruct wedge_graph {")]
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).strip().encode())
    return h.hexdigest()[:16]


def _traffic(key):
    val, _, digest = TRAFFIC[key]
    return val if val is not None and digest == _kernel_digest(key) else None


def _ncu_gbs(key):
    """DRAM bytes over the launch's duration, both from the ncu capture."""
    val, us, digest = TRAFFIC[key]
    return val / (us * 1e-6) / 1e9 if val is not None and digest == _kernel_digest(key) else None


def _gather_bound(torch, dev, edges, t, clocks, probe_t=None, lib_t=None):
    """Every edge costs one random gather, and each distinct 128-byte line a
    gather instruction touches is one L1 wavefront; the L1 data pipe retires
    one wavefront per clock per SM (ncu: l1tex__data_pipe_lsu_wavefronts).
    probe_t: the shortest time of the probe (libwedge_probe.so) over the same
    edges (the same source stream and gathers without the reduction), a
    measured ceiling of this access pattern.  lib_t: the shortest time of a
    library gather of the same values by the same sources
    (torch.index_select with the int32 source array as index), a ceiling
    measured with code and a launch shape that are not this project's."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = sms * mhz * 1e6 / 1e9
    achieved = edges / t / 1e9
    out = {"unit": "G gathers/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
           "peak_basis": f"{sms} SMs x {mhz:.0f} MHz x 1 L1 wavefront/clock"}
    if probe_t:
        out.update({"measured_peak": edges / probe_t / 1e9, "frac_of_measured": probe_t / t,
                    "measured_peak_basis": "wedge_probe_gather: the pull's 16-byte source stream and one 4-byte "
                                           "gather per edge, no reduction, same launch shape"})
    if lib_t:
        out.update({"library_gather": edges / lib_t / 1e9, "frac_of_library_gather": lib_t / t,
                    "library_gather_basis": "torch.index_select(values, 0, int32 sources, out=...): reads the "
                                            "sources, gathers one 4-byte value per edge and writes it out; "
                                            "best of 20"})
    return out


def gather_ceilings(torch, stream, src, E, vals):
    """Shortest times (s) over 20 launches of the probe and of the library
    gather, both over `src` (int32 device tensor of E sources) into `vals`."""
    from paper_1903_07754_gb300 import probe
    sink = torch.zeros(1, dtype=torch.float32, device=vals.device)
    tp = _time_launch(torch, stream, lambda: probe.wedge_probe_gather(src, E, vals, sink, stream=stream), reps=20,
                      warm=3, best=True)
    buf = torch.empty(E, dtype=torch.float32, device=vals.device)
    idx = src[:E]

    def lib():
        with torch.cuda.stream(stream):
            torch.index_select(vals, 0, idx, out=buf)

    tl = _time_launch(torch, stream, lib, reps=20, warm=3, best=True)
    return tp, tl


def _time_launch(torch, stream, fn, before=None, reps=10, warm=2, best=False):
    """Mean (or, with best, the shortest) device time (s) of fn() per
    CUDA-event pair on `stream`."""
    times = []
    for r in range(reps + warm):
        if before:
            before()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= warm:
            times.append(e0.elapsed_time(e1))
    return (float(np.min(times)) if best else float(np.mean(times))) / 1e3


def roofline_pr_pull(wedge, torch, G, g, stream, dev, clocks):
    """PageRank's dense pull (k_pull<PR>) on the contributions of pr0 as a
    PageRank run executes it: contributions in the run's gather order
    (`wedge_pr_order`, arranged outside the timed region) through
    `wedge_pr_pull_ordered`, one launch per CUDA-event pair (the sums are
    zeroed outside the pair).  The measured gather ceilings read the same
    renamed sources and ordered contributions."""
    V, E = g.V, g.E
    od = torch.from_numpy(g.outdeg().astype(np.float32)).to(dev)
    contrib = torch.where(od > 0, (1.0 / V) / torch.clamp(od, min=1.0), torch.zeros_like(od)).contiguous()
    order = torch.empty(V, dtype=torch.int32, device=dev)
    wedge.wedge_pr_order(G.handle, order)
    ordered = torch.empty_like(contrib)
    ordered[order.long()] = contrib
    sums = torch.zeros(V, dtype=torch.int64, device=dev)
    times = []
    for r in range(12):
        sums.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wedge.wedge_pr_pull_ordered(G.handle, ordered, sums)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    t = float(np.mean(times)) / 1e3
    # algorithmic bytes: offsets 4(V+1), sources 4E, each contribution
    # gathered once 4V (V*4 <= L2), 64-bit fixed-point sums written 8V; the
    # other count takes every gather as one 32-byte sector
    alg = 4 * (V + 1) + 4 * E + 4 * V + 8 * V
    alg_sectors = 4 * (V + 1) + 4 * E + 32 * E + 8 * V
    src_ordered = order[G.device_src.long()].contiguous()  # the run's renamed sources
    tp, tl = gather_ceilings(torch, stream, src_ordered, E, ordered)
    del src_ordered
    return _roofline("k_pull<PR> dense (PageRank in-edge pass, R-MAT s22, gather order)", "pr", alg, alg_sectors, t,
                     dev, _gather_bound(torch, dev, E, t, clocks, tp, tl))


def _roofline(kernel, key, alg, alg_sectors, t, dev, gather):
    import torch
    peak, kind = peaks()
    achieved = alg / t / 1e9
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": kind,
            "unit": "GB/s", "frac": achieved / peak, "traffic": _traffic(key), "alg_bytes": alg, "ms": t * 1e3,
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
            "gathers_counted": f"once per vertex (V*4 <= L2 = {l2 >> 20} MB)",
            "alg_bytes_gather_sectors": alg_sectors, "achieved_gather_sectors": alg_sectors / t / 1e9,
            "ncu_dram_gbs": _ncu_gbs(key), "gather_bound": gather}


def transform_case(wedge, torch, G, g, od, stream, dev, frac=0.10, seed=5):
    """One frontier transformation (wedge_frontier_transform, k = 0) of a
    seeded random frontier holding `frac` of the vertices: its time and its
    algorithmic bytes -- the frontier bitmap V/8, two row offsets per active
    vertex, the rows' entries, the Wedge bitmap NC/8 and the list."""
    rng = np.random.default_rng(seed)
    mask = rng.random(g.V) < frac
    packed = np.packbits(mask, bitorder="little")
    packed = np.concatenate([packed, np.zeros((-packed.size) % 4, dtype=np.uint8)])
    bm = torch.from_numpy(packed.view(np.int32).copy()).to(dev)
    nc = (g.E + 31) // 32
    clist = torch.empty(nc, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    t = _time_launch(torch, stream, lambda: wedge.wedge_frontier_transform(G.handle, bm, 0, clist, cnt), reps=10)
    eo = np.empty(g.V + 1, dtype=np.uint32)
    d_eo = torch.empty(g.V + 1, dtype=torch.int32, device=dev)
    info = wedge.wedge_graph_get_info(G.handle)
    d_ei = torch.empty(max(info["eidx_len"], 1), dtype=torch.int32, device=dev)
    wedge.wedge_graph_copy_edge_index(G.handle, d_eo, d_ei)
    eo[:] = d_eo.cpu().numpy().view(np.uint32)
    rows = int((eo[1:].astype(np.int64) - eo[:-1])[mask].sum())
    entries = int(cnt.item())
    alg = g.V / 8 + 8 * int(mask.sum()) + 4 * rows + nc / 8 + 4 * entries
    return {"frontier": int(mask.sum()), "row_entries": rows, "list_entries": entries, "ms": t * 1e3,
            "alg_bytes": alg, "alg_gbs": alg / t / 1e9, "entries_per_s": rows / t}


def compressed_index(wedge, torch, G, g, od, stream, dev, sssp_opts):
    """The compressed edge index on the benchmark graph: its size against the
    plain index, its build time, and the 10% transformation and the SSSP run
    with each index (the transformation's algorithmic bytes count the index
    entries it reads: 4 per entry plain; header + packed words compressed)."""
    info0 = wedge.wedge_graph_get_info(G.handle)
    plain = transform_case(wedge, torch, G, g, od, stream, dev)
    dist = torch.empty(g.V, dtype=torch.int32, device=dev)
    t_sssp = _time_launch(torch, stream, lambda: wedge.wedge_run_sssp(G.handle, 0, dist, sssp_opts, False), reps=10)
    before = wedge.wedge_graph_get_tuning(G.handle)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    wedge.wedge_graph_set_tuning(G.handle, before["dense_loader"], before["blocks_per_sm"], 1)
    build_ms = (time.perf_counter() - t0) * 1e3
    info1 = wedge.wedge_graph_get_info(G.handle)
    comp = transform_case(wedge, torch, G, g, od, stream, dev)
    t_sssp_z = _time_launch(torch, stream, lambda: wedge.wedge_run_sssp(G.handle, 0, dist, sssp_opts, False),
                            reps=10)
    wedge.wedge_graph_set_tuning(G.handle, before["dense_loader"], before["blocks_per_sm"], before["edge_index"])
    ratio = info1["eidx_z_bytes"] / info0["eidx_bytes"]
    return {"plain_bytes": info0["eidx_bytes"], "compressed_bytes": info1["eidx_z_bytes"], "ratio": ratio,
            "build_ms": build_ms, "transform10_ms": {"plain": plain["ms"], "compressed": comp["ms"]},
            "transform10_index_bytes": {"plain": 4 * plain["row_entries"],
                                        "compressed_est": ratio * 4 * plain["row_entries"]},
            "sssp_ms": {"plain": t_sssp * 1e3, "compressed": t_sssp_z * 1e3}}


def balance_summary(rec, kernel):
    """Busy and idle shares of one transformation kernel's warps (Fig. 13's
    division of thread time): a warp is busy from its start to the end of its
    last piece, idle from then to the kernel's last end; the span runs from
    the first start to the last end."""
    r = rec[:, kernel, :].astype(np.float64)
    start, end, cyc = r[:, 0], r[:, 1], r[:, 2]
    span = end.max() - start.min()
    busy = end - start
    return {"span_us": span / 1e3, "busy_mean_us": busy.mean() / 1e3, "busy_max_us": busy.max() / 1e3,
            "idle_frac": float(1.0 - busy.sum() / (r.shape[0] * span)) if span > 0 else 0.0,
            "busy_max_over_mean": float(busy.max() / busy.mean()) if busy.mean() > 0 else 1.0,
            "cycles_max_over_mean": float(cyc.max() / cyc.mean()) if cyc.mean() > 0 else 1.0}


def transform_balance(wedge, torch, G, g, stream, dev):
    """Load balance of the frontier transformation (Section 5.3, Fig. 13) on
    two frontiers of the benchmark graph: a seeded random 10% of the vertices
    and SSSP's frontier after four dense pulls from vertex 0; under the
    library's schedule (rows cut into 32-entry pieces, balanced expansion)
    and the paper's (equal slices of the vertex frontier, whole rows per
    warp).  Per schedule: the call's device time and each kernel's idle
    share of warp time."""
    V = g.V
    words = (V + 31) // 32
    rng = np.random.default_rng(5)
    packed = np.packbits(rng.random(V) < 0.10, bitorder="little")
    packed = np.concatenate([packed, np.zeros((-packed.size) % 4, dtype=np.uint8)])
    fronts = {"random10": torch.from_numpy(packed.view(np.int32).copy()).to(dev)}
    vals = torch.full((V,), -1, dtype=torch.int32, device=dev)
    vals[0] = 0
    nxt = torch.zeros(words, dtype=torch.int32, device=dev)
    full = torch.zeros(1, dtype=torch.int64, device=dev)
    nf = torch.zeros(1, dtype=torch.int32, device=dev)
    for t in range(4):
        nxt.zero_()
        wedge.wedge_pull_iterate(G.handle, "sssp", vals, t, None, None, None, 0, nxt, full, nf)
    fronts["sssp_iter4"] = nxt.clone()
    nc = (g.E + 31) // 32
    clist = torch.empty(nc, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {}
    for name, bm in fronts.items():
        res = {"frontier": int(np.unpackbits(bm.cpu().numpy().view(np.uint8)).sum())}
        for sched in (0, 1):
            rec = None
            for _ in range(3):
                rec = wedge.wedge_frontier_transform_profile(G.handle, bm, 0, sched, clist, cnt)
            # the library's schedule through its plain entry point; the
            # paper's exists only in the profiling call (whose record copy
            # adds a little host time to its 5 ms)
            t = _time_launch(torch, stream, (lambda: wedge.wedge_frontier_transform(G.handle, bm, 0, clist, cnt))
                             if sched == 0 else (lambda: wedge.wedge_frontier_transform_profile(
                                 G.handle, bm, 0, sched, clist, cnt)), reps=5)
            kern = {"scan": balance_summary(rec, 0), "expand": balance_summary(rec, 1)} if sched == 0 else \
                {"slices": balance_summary(rec, 0)}
            span = sum(k["span_us"] for k in kern.values())
            res["library" if sched == 0 else "paper_static_slices"] = {"ms": t * 1e3, "kernels": kern,
                                                                       "kernel_span_us": span}
            res["list_entries"] = int(cnt.item())
        res["speedup_library_vs_paper"] = res["paper_static_slices"]["ms"] / res["library"]["ms"]
        res["speedup_library_vs_paper_kernel_span"] = (res["paper_static_slices"]["kernel_span_us"] /
                                                       res["library"]["kernel_span_us"])
        out[name] = res
    return out


def roofline_dense_pull(wedge, torch, G, S, g, s, stream, dev):
    """Dense CC pull on the symmetric graph from the initial labels (every
    destination changes), one launch per CUDA-event pair."""
    V, E = s.V, s.E
    init = torch.arange(V, dtype=torch.int32, device=dev)
    vals = torch.empty_like(init)
    words = (V + 31) // 32
    nxt = torch.zeros(words, dtype=torch.int32, device=dev)
    full = torch.zeros(1, dtype=torch.int64, device=dev)
    nf = torch.zeros(1, dtype=torch.int32, device=dev)
    times = []
    for r in range(12):
        vals.copy_(init)
        nxt.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wedge.wedge_pull_iterate(S.handle, "cc", vals, 0, None, None, None, 0, nxt, full, nf)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    t = float(np.mean(times)) / 1e3
    nchanged = int(nf.item())
    # algorithmic bytes of one dense CC pull: offsets 4(V+1), sources 4E, each
    # label gathered once 4V (V*4 <= L2), destination labels read 4V,
    # changed labels written 4*changed, next-frontier bitmap V/8
    alg = 4 * (V + 1) + 4 * E + 4 * V + 4 * V + 4 * nchanged + V / 8
    alg_sectors = 4 * (V + 1) + 4 * E + 32 * E + 4 * V + 4 * nchanged + V / 8
    fv = torch.rand(V, dtype=torch.float32, device=dev)
    tp, tl = gather_ceilings(torch, stream, S.device_src, E, fv)
    return _roofline("k_pull<CC> dense (first CC iteration, R-MAT s22 sym)", "cc", alg, alg_sectors, t, dev,
                     _gather_bound(torch, dev, E, t, None, tp, tl))


def e2e_measure(wedge, torch, g, s, od, edges, args, dev, opts):
    """Host buffers through the public API: pinned host CSC -> device, graph
    creation (edge index build), the four runs, results back to the host.
    Three streams: the R-MAT graph's CSC copy, creation and BFS/SSSP/
    PageRank runs on one; its weights' copy on another, beside the creation
    (SSSP waits for it); the symmetrised graph's copies (queued behind the
    weights), creation and CC on a third, overlapping the first."""
    host = {}
    for name, arr in (("off", g.offsets), ("src", g.src), ("w", g.w), ("soff", s.offsets), ("ssrc", s.src)):
        t = torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)).pin_memory()
        host[name] = t
    h2d = sum(t.numel() * 4 for t in host.values())
    outs = {n: torch.empty(g.V, dtype=torch.int32).pin_memory() for n in ("lvl", "lab", "dist")}
    outs["pr"] = torch.empty(g.V, dtype=torch.float32).pin_memory()
    d2h = sum(t.numel() * 4 for t in outs.values())
    stream = torch.cuda.current_stream()
    sa, sb, sw = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def one():
        for st in (sa, sb, sw):
            st.wait_stream(stream)
        # the host link carries one copy at a time at full rate: the R-MAT
        # CSC first, then its weights (creation does not read them), then
        # the symmetrised CSC
        with torch.cuda.stream(sa):
            dg = {n: host[n].to(dev, non_blocking=True) for n in ("off", "src")}
            csc_copied = torch.cuda.Event()
            csc_copied.record(sa)
        with torch.cuda.stream(sw):
            sw.wait_event(csc_copied)
            dg["w"] = host["w"].to(dev, non_blocking=True)
            w_copied = torch.cuda.Event()
            w_copied.record(sw)
        with torch.cuda.stream(sb):
            sb.wait_event(w_copied)
            ds = {n: host[n].to(dev, non_blocking=True) for n in ("soff", "ssrc")}
        with torch.cuda.stream(sa):
            G = wedge.Graph(wedge.wedge_graph_create(g.V, g.E, dg["off"], dg["src"], dg["w"]), keep=list(dg.values()))
            lvl = torch.empty(g.V, dtype=torch.int32, device=dev)
            dst = torch.empty_like(lvl)
            pr = torch.empty(g.V, dtype=torch.float32, device=dev)
            wedge.wedge_run_bfs(G.handle, 0, lvl, opts[0], False)
            sa.wait_event(w_copied)  # SSSP reads the weights
            wedge.wedge_run_sssp(G.handle, 0, dst, opts[2], False)
            wedge.wedge_run_pr(G.handle, pr, PR_ITERS, DAMPING, None, False)
            outs["lvl"].copy_(lvl, non_blocking=True)
            outs["dist"].copy_(dst, non_blocking=True)
            outs["pr"].copy_(pr, non_blocking=True)
        with torch.cuda.stream(sb):
            S = wedge.Graph(wedge.wedge_graph_create(s.V, s.E, ds["soff"], ds["ssrc"]), keep=list(ds.values()))
            lab = torch.empty(s.V, dtype=torch.int32, device=dev)
            wedge.wedge_run_cc(S.handle, lab, opts[1], False)
            outs["lab"].copy_(lab, non_blocking=True)
        for st in (sa, sb, sw):
            stream.wait_stream(st)
        torch.cuda.synchronize()
        G.close()
        S.close()

    one()
    times = []
    for _ in range(5):  # median of five end-to-end steps, each between CUDA events
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    return {"value": sum(edges.values()) / (ms / 1e3) / 1e9, "unit": "GTEPS", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "includes": "H2D of both CSCs, two wedge_graph_create (edge index build), 4 runs, D2H of results; "
                        "the weights' copy beside the R-MAT graph's creation, the symmetrised graph's copies, "
                        "creation and CC on other streams"}


def cpu_baseline(g, s, od):
    """The oracle as it stands, single-threaded on the host, on a bounded
    sample of the step: BFS, CC and PageRank (2 of the 20 iterations) on the
    full graphs; SSSP (Dijkstra) on the full graph."""
    import oracle
    t0 = time.perf_counter()
    lvl = oracle.bfs_push(g, 0)
    t1 = time.perf_counter()
    oracle.cc_union_find(s)
    t2 = time.perf_counter()
    dist = oracle.sssp_dijkstra(g, 0)
    t3 = time.perf_counter()
    oracle.pr_pull(g, DAMPING, 2)
    t4 = time.perf_counter()
    edges = credited_edges(od, lvl != 0xFFFFFFFF) + s.E + credited_edges(od, dist != 0xFFFFFFFF) + 2 * g.E
    secs = t4 - t0
    return {"value": edges / secs / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": "full-size BFS (push), CC (union-find), SSSP (Dijkstra) and 2 of 20 PageRank "
                      f"iterations (FP64 pull) on the same graphs; {secs:.1f} s on 1 host core",
            "seconds": {"bfs": t1 - t0, "cc": t2 - t1, "sssp": t3 - t2, "pr2": t4 - t3},
            "host_cores_available": os.cpu_count(), "all_cores": cpu_baseline_all_cores(g, s, od)}


def cpu_baseline_all_cores(g, s, od):
    """The oracle's pull variants with their destination loop shared among
    every host core (OpenMP; the same results as the single-threaded pulls):
    BFS, CC (HCC) and SSSP (Bellman-Ford) by dense pulls until the frontier
    is empty, and 2 of the 20 PageRank iterations; the median of 3 runs of
    each, credited with the step's edges."""
    import oracle
    secs = {}
    lvl = dist = None
    for name, fn in (("bfs", lambda: oracle.dense_pull_omp("bfs", g, 0)),
                     ("cc", lambda: oracle.dense_pull_omp("cc", s, 0)),
                     ("sssp", lambda: oracle.dense_pull_omp("sssp", g, 0)),
                     ("pr2", lambda: oracle.pr_pull_omp(g, DAMPING, 2))):
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            r = fn()
            ts.append(time.perf_counter() - t0)
        secs[name] = float(np.median(ts))
        if name == "bfs":
            lvl = r[0]
        elif name == "sssp":
            dist = r[0]
    edges = credited_edges(od, lvl != 0xFFFFFFFF) + s.E + credited_edges(od, dist != 0xFFFFFFFF) + 2 * g.E
    total = sum(secs.values())
    return {"value": edges / total / 1e9, "unit": "GTEPS", "cores": oracle.omp_threads(), "kind": "oracle",
            "sample": "dense pulls (BFS, HCC, Bellman-Ford until the frontier is empty) and 2 of 20 PageRank "
                      f"iterations, destinations shared among {oracle.omp_threads()} threads; median of 3 runs "
                      f"each, {total:.2f} s", "seconds": secs}


if __name__ == "__main__":
    main()
