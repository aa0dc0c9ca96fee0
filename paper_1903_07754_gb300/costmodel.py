"""Learned switch: trace collection, GPU training and evaluation of the cost
model (not in the paper; it replaces the fixed fullness threshold and the
fixed Wedge Frontier precision of Section 3.4).

Every step runs in the library's kernels: traces come from
`wedge_trace_candidates` (each candidate timed from the same saved state),
training uses `wedge_mlp_loss_grad` and `wedge_mlp_adam` on device tensors,
and choices are made by `wedge_mlp_forward_bf16`, the same BF16 arithmetic as
the in-loop decision.
"""
from __future__ import annotations

import os

import numpy as np

from . import wedge

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "cost_model.npy")


def collect(handle, app, roots, opts=None, max_iters=256, cap=4096):
    """Traces of `app` from each root: list of (features [n,6,12], ms [n,6],
    threshold choice [n])."""
    out = []
    if opts is not None and opts.log2_coarsen > 7:
        # the candidates are dense and k = 0..4: trace at chunk precision
        import copy
        opts = copy.copy(opts)
        opts.log2_coarsen = 0
    for r in roots:
        feat, ms, chosen = wedge.wedge_trace_candidates(handle, app, int(r), opts, max_iters, cap)
        if len(ms):
            out.append((feat, ms, chosen))
    return out


def dataset(traces):
    """Training rows: features -> ln(ms) of every timed candidate."""
    X = np.concatenate([f.reshape(-1, wedge.MLP_FEATURES) for f, _, _ in traces]).astype(np.float32)
    T = np.log(np.maximum(np.concatenate([m.reshape(-1) for _, m, _ in traces]), 1e-4)).astype(np.float32)
    return X, T


def init_params(seed=0):
    """He-initialised weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(wedge.MLP_PARAMS, dtype=np.float32)
    p[0:768] = rng.normal(0, np.sqrt(2.0 / 12), 768)
    p[832:4928] = rng.normal(0, np.sqrt(2.0 / 64), 4096)
    p[4992:5056] = rng.normal(0, np.sqrt(1.0 / 64), 64)
    return p


def train(X, T, steps=1500, lr=3e-3, seed=0, params=None, log_every=0):
    """Full-batch Adam on the GPU with the library's kernels.  Returns
    (params as numpy FP32, final loss)."""
    import torch
    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
    p = torch.from_numpy(init_params(seed) if params is None else np.array(params, dtype=np.float32)).to(dev)
    g = torch.zeros_like(p)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    n = x.shape[0]
    last = None
    for step in range(1, steps + 1):
        wedge.wedge_mlp_loss_grad(p, x, t, n, g, loss)
        wedge.wedge_mlp_adam(p, g, m, v, step, lr)
        if log_every and step % log_every == 0:
            print(f"step {step} loss {loss.item():.5f}", flush=True)
    wedge.wedge_mlp_loss_grad(p, x, t, n, g, loss)
    last = float(loss.item())
    return p.cpu().numpy(), last


def predict_bf16(params, feats):
    """Predicted ln(ms) for every candidate row, as the decision computes it."""
    import torch
    f = np.ascontiguousarray(feats.reshape(-1, wedge.MLP_FEATURES), dtype=np.float32)
    x = torch.from_numpy(f).cuda()
    y = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    wedge.wedge_mlp_forward_bf16(p, x, x.shape[0], y)
    return y.cpu().numpy().reshape(feats.shape[:-1])


def choose(params, feats):
    return np.argmin(predict_bf16(params, feats), axis=-1)


def regret(ms, choice):
    """Sum over iterations of the chosen candidate's time minus the best."""
    ms = np.asarray(ms)
    return float((ms[np.arange(len(ms)), choice] - ms.min(axis=1)).sum())


NO_BAND = (0.0, 3.0e38)


def learn_band(traces, pad=2.0, rtol=0.05, atol_ms=0.002, quantile=0.0):
    """The band of fullness / E (feature 3) outside which one candidate was,
    within timing noise (rtol of the fastest plus atol_ms), the fastest at
    every traced iteration (all but a `quantile` share of them at each end):
    below lo the Wedge Frontier at k = 0 (candidate 1), above hi a dense
    pull (candidate 0).  Widened by `pad` on both sides; the decision
    evaluates the model only inside it."""
    x = np.concatenate([f[:, 0, 2] for f, _, _ in traces]).astype(np.float64)
    ms = np.concatenate([m for _, m, _ in traces])
    tol = ms.min(axis=1) * (1 + rtol) + atol_ms
    sparse0_slow = ms[:, 1] > tol   # iterations where k = 0 was clearly not the fastest
    dense_slow = ms[:, 0] > tol     # ... where a dense pull was clearly not
    lo = float(np.quantile(x[sparse0_slow], quantile)) / pad if np.any(sparse0_slow) else NO_BAND[1]
    hi = float(np.quantile(x[dense_slow], 1.0 - quantile)) * pad if np.any(dense_slow) else 0.0
    if hi < lo:  # the regions meet: no fullness needs the model
        lo = hi = (lo + hi) / 2 if lo < NO_BAND[1] else hi
    return lo, hi


def choose_in_band(params, feats, band=NO_BAND):
    """The decision's choice with the band: the model inside it, candidate 1
    below it, candidate 0 above it."""
    x = feats[:, 0, 2]
    c = choose(params, feats)
    return np.where(x < band[0], 1, np.where(x > band[1], 0, c))


def evaluate(params, traces, band=NO_BAND):
    """(learned regret, threshold regret, best possible total ms)."""
    lr_, th = 0.0, 0.0
    best = 0.0
    for feat, ms, chosen in traces:
        lr_ += regret(ms, choose_in_band(params, feat, band))
        th += regret(ms, chosen.astype(np.int64))
        best += float(ms.min(axis=1).sum())
    return lr_, th, best


def save(params, path=DEFAULT_MODEL):
    np.save(path, np.asarray(params, dtype=np.float32))


def load_params(path=DEFAULT_MODEL):
    p = np.load(path)
    if p.shape != (wedge.MLP_PARAMS,):
        raise ValueError("cost model must hold 5057 parameters")
    return p.astype(np.float32)


def load_band(path=None):
    """The band saved beside the model (cost_model.json's "band"), or no band."""
    import json
    path = path or os.path.join(os.path.dirname(DEFAULT_MODEL), "cost_model.json")
    try:
        with open(path) as f:
            lo, hi = json.load(f)["band"]
        return float(lo), float(hi)
    except (OSError, KeyError, ValueError):
        return NO_BAND
