"""Learned switch on the GPU: the cost model's kernels against the FP64
oracle element by element (FP32 forward, BF16 forward, gradient, Adam),
the candidate-timing traces, end-to-end correctness of learned runs,
and what the trained model gains over the fixed threshold."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from oracle import mlp as omlp
from _gpu import empty_u32, graph, opts, u32
from paper_1903_07754_gb300 import costmodel, wedge

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(seed, n):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, omlp.NPARAMS).astype(np.float32)
    X = rng.uniform(0, 1, (n, omlp.IN)).astype(np.float32)
    T = rng.normal(0, 1, n).astype(np.float32)
    return p, X, T


@pytest.mark.parametrize("n", [1, 77, 300, 1000])
def test_gradient_matches_oracle(n):
    """Every component of the FP32 gradient against the FP64 oracle's:
    |g_i - o_i| <= 1e-3 |o_i| + 1e-6 max_j |o_j| (a small block such as b3 or
    w3 is held to its own size, not hidden under W2's norm)."""
    p, X, T = _case(n, n)
    g = torch.empty(omlp.NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    wedge.wedge_mlp_loss_grad(_t(p), _t(X), _t(T), n, g, loss)
    L, gw = omlp.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.item() - L) <= 1e-4 * max(1.0, abs(L))
    got = g.cpu().numpy().astype(np.float64)
    tol = 1e-3 * np.abs(gw) + 1e-6 * np.abs(gw).max()
    bad = np.flatnonzero(np.abs(got - gw) > tol)
    assert bad.size == 0, (bad[:10], got[bad[:10]], gw[bad[:10]])
    # each block of the layout carries gradient (the case exercises them all)
    for lo, hi in ((omlp.W1, omlp.B1), (omlp.B1, omlp.W2), (omlp.W2, omlp.B2), (omlp.B2, omlp.W3),
                   (omlp.W3, omlp.B3), (omlp.B3, omlp.NPARAMS)):
        assert np.any(gw[lo:hi] != 0.0)


def test_adam_matches_oracle_elementwise():
    """wedge_mlp_adam against the FP64 Adam step after 1, 2 and 50 steps of
    the same seeded gradients.  Scales: the moving averages of |g| and g^2
    (FP32 keeps ~1e-7 of them per step, plus the FP32 rounding of the
    betas) and the sum of the oracle's step sizes (the update's FP32
    arithmetic, including the host's beta^t, keeps ~1e-5 of each step)."""
    rng = np.random.default_rng(17)
    n, lr = omlp.NPARAMS, 2e-3
    G = rng.normal(0, 1, (50, n)).astype(np.float32)
    G[:, ::7] *= 1e-3   # small gradients too
    p0 = rng.normal(0, 0.3, n).astype(np.float32)
    dp, dm, dv = _t(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    op, om, ov = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    abs_m, moved = np.zeros(n), np.zeros(n)
    for t in range(1, 51):
        wedge.wedge_mlp_adam(dp, _t(G[t - 1]), dm, dv, t, lr)
        prev = op
        op, om, ov = omlp.adam_step(op, G[t - 1].astype(np.float64), om, ov, t, lr)
        abs_m = 0.9 * abs_m + 0.1 * np.abs(G[t - 1])
        moved += np.abs(op - prev)
        if t in (1, 2, 50):
            gp, gm, gv = (x.cpu().numpy().astype(np.float64) for x in (dp, dm, dv))
            assert np.all(np.abs(gm - om) <= 1e-5 * abs_m), f"m, step {t}"
            # v: (1 - beta2) in FP32 is 1 - 0.999f = 0.00099998713, 1.3e-5
            # below 0.001, so every FP32 second moment sits ~1.3e-5 low
            assert np.all(np.abs(gv - ov) <= 3e-5 * ov), f"v, step {t}"
            tol = 1e-4 * moved + 2 * t * 2.0 ** -24 * np.abs(op)
            bad = np.flatnonzero(np.abs((gp - p0) - (op - p0)) > tol)
            assert bad.size == 0, (t, bad[:10], gp[bad[:10]], op[bad[:10]])


def test_forward_fp32_and_bf16_match_oracle():
    p, X, _ = _case(7, 513)
    y = torch.empty(513, dtype=torch.float32, device="cuda")
    wedge.wedge_mlp_forward(_t(p), _t(X), 513, y)
    want = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), want, rtol=1e-5, atol=1e-5)
    wedge.wedge_mlp_forward_bf16(_t(p), _t(X), 513, y)
    got = y.cpu().numpy().astype(np.float64)
    want16 = omlp.forward_bf16(p, X)
    # The kernel sums BF16 products in FP32, the oracle in FP64: the sums
    # agree to ~1e-6 of the sum of |terms| (`scale`), unless a hidden
    # pre-activation lies that close to a BF16 rounding boundary and rounds
    # the other way: then one activation moves by one BF16 step, at most
    # 2^-7 of its value.  `flips`: every hidden unit of both layers moving by
    # one step at once (layer-1 steps carried through |W2| and |w3|), a
    # bound no row may pass; almost every row must match to 1e-5 of scale.
    w1, b1, w2, b2, w3, b3 = (omlp.bf16(np.asarray(a, dtype=np.float32)).astype(np.float64)
                              for a in omlp.unpack(p))
    x = omlp.bf16(X).astype(np.float64)
    h1 = omlp.bf16(np.maximum(x @ w1.T + b1, 0.0)).astype(np.float64)
    h2 = omlp.bf16(np.maximum(h1 @ w2.T + b2, 0.0)).astype(np.float64)
    scale = np.abs(h2) @ np.abs(w3) + abs(b3)
    flips = 2.0 ** -7 * (np.abs(h2) @ np.abs(w3) + (np.abs(h1) @ np.abs(w2).T) @ np.abs(w3))
    diff = np.abs(got - want16)
    assert np.all(diff <= flips + 1e-5 * scale)
    assert np.mean(diff <= 1e-5 * scale) >= 0.97, np.mean(diff <= 1e-5 * scale)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (2000, 12)).astype(np.float32)
    T = (np.log1p(X[:, 0] * 10) + X[:, 1] - 0.5 * X[:, 10]).astype(np.float32)
    p0 = costmodel.init_params(0)
    l0 = omlp.loss(p0, X, T)
    p, l1 = costmodel.train(X, T, steps=600, lr=3e-3)
    assert l1 < 0.05 * l0
    assert abs(l1 - omlp.loss(p, X, T)) <= 1e-3 * max(l1, 1e-3) + 1e-5


@pytest.fixture(scope="module")
def g16():
    return gg.rmat(16, 16).with_weights(255)


def test_trace_candidates_follow_the_threshold(g16):
    G = graph(g16)
    try:
        tau, k = 500, 2
        o = opts("bfs", tau=tau, k=k)
        feat, ms, chosen = wedge.wedge_trace_candidates(G.handle, "bfs", 0, o)
        _, ot = oracle.wedge_run("bfs", g16, 0, oracle.POLICY_THRESHOLD, tau, 32 << k)
        assert len(ms) == ot.shape[0]
        assert np.all(ms > 0) and np.all(np.isfinite(feat))
        np.testing.assert_array_equal(chosen, np.where(ot[:, 2] == 1, k + 1, 0))
        # features 11-12 encode the candidate; 1-2 the frontier
        np.testing.assert_array_equal(feat[0, :, 10], [0, 1, 1, 1, 1, 1])
        np.testing.assert_allclose(feat[:, 0, 0], np.log2(ot[:, 0] + 1.0) / 32, rtol=1e-6)
        # after tracing, a normal run still matches the oracle
        out = empty_u32(g16.V)
        wedge.wedge_run_bfs(G.handle, 0, out)
        np.testing.assert_array_equal(u32(out)[: g16.V], oracle.bfs_push(g16, 0))
    finally:
        G.close()


def _traces(specs):
    traces = []
    for scale, a, seed in specs:
        b = (1 - a) * 0.19 / 0.43
        g = gg.rmat(scale, 16, a=a, b=b, c=b, seed=seed).with_weights(255)
        s = gg.symmetrize(gg.Graph(g.V, g.offsets, g.src))
        G, S = graph(g), graph(s, with_weights=False)
        roots = gg.roots(g, 2, seed=seed)
        traces += costmodel.collect(G.handle, "bfs", roots, opts("bfs"), 64)
        traces += costmodel.collect(G.handle, "sssp", roots[:1], opts("sssp"), 64)
        traces += costmodel.collect(S.handle, "cc", [0], opts("cc"), 64)
        G.close()
        S.close()
    return traces


def test_learned_switch_gains_over_threshold_and_stays_exact(g16):
    train_tr = _traces([(16, 0.45, 11), (16, 0.57, 12), (16, 0.70, 13), (17, 0.57, 14)])
    test_tr = _traces([(16, 0.57, 21), (17, 0.50, 22)])
    X, T = costmodel.dataset(train_tr)
    params, loss = costmodel.train(X, T, steps=2000, lr=3e-3)
    learned, threshold, best = costmodel.evaluate(params, test_tr)
    band = costmodel.learn_band(train_tr)
    learned_band, _, _ = costmodel.evaluate(params, test_tr, band)
    print(f"held-out regret: learned {learned:.3f} ms (with band {band}: {learned_band:.3f} ms), "
          f"threshold {threshold:.3f} ms, best total {best:.3f} ms, train loss {loss:.4f}")
    assert learned <= threshold
    assert learned_band <= threshold
    # learned runs reach the exact results, with and without the band
    G = graph(g16)
    try:
        wedge.wedge_set_cost_model(G.handle, params)
        wedge.wedge_set_learned_band(G.handle, *band)
        out = empty_u32(g16.V)
        o = opts("bfs", switch=wedge.SWITCH_LEARNED)
        st = wedge.wedge_run_bfs(G.handle, 0, out, o)
        np.testing.assert_array_equal(u32(out)[: g16.V], oracle.bfs_push(g16, 0))
        o = opts("sssp", switch=wedge.SWITCH_LEARNED)
        wedge.wedge_run_sssp(G.handle, 0, out, o)
        np.testing.assert_array_equal(u32(out)[: g16.V], oracle.sssp_dijkstra(g16, 0))
        assert st.iters > 0
        wedge.wedge_set_learned_band(G.handle, *costmodel.NO_BAND)
        wedge.wedge_run_sssp(G.handle, 0, out, o)
        np.testing.assert_array_equal(u32(out)[: g16.V], oracle.sssp_dijkstra(g16, 0))
        with pytest.raises(wedge.WedgeError):
            wedge.wedge_set_learned_band(G.handle, 0.5, 0.1)
    finally:
        G.close()
