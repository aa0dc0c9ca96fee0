"""Learned switch on the GPU: the cost model's kernels against the FP64
oracle, the candidate-timing traces, end-to-end correctness of learned runs,
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
    p, X, T = _case(n, n)
    g = torch.empty(omlp.NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    wedge.wedge_mlp_loss_grad(_t(p), _t(X), _t(T), n, g, loss)
    L, gw = omlp.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.item() - L) <= 1e-4 * max(1.0, abs(L))
    got = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - gw) <= 1e-3 * np.linalg.norm(gw)


def test_forward_fp32_and_bf16_match_oracle():
    p, X, _ = _case(7, 513)
    y = torch.empty(513, dtype=torch.float32, device="cuda")
    wedge.wedge_mlp_forward(_t(p), _t(X), 513, y)
    want = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), want, rtol=1e-5, atol=1e-5)
    wedge.wedge_mlp_forward_bf16(_t(p), _t(X), 513, y)
    want16 = omlp.forward_bf16(p, X)
    np.testing.assert_allclose(y.cpu().numpy(), want16, rtol=2e-2, atol=2e-2)


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
    print(f"held-out regret: learned {learned:.3f} ms, threshold {threshold:.3f} ms, best total {best:.3f} ms, "
          f"train loss {loss:.4f}")
    assert learned <= threshold
    # learned runs reach the exact results
    G = graph(g16)
    try:
        wedge.wedge_set_cost_model(G.handle, params)
        out = empty_u32(g16.V)
        o = opts("bfs", switch=wedge.SWITCH_LEARNED)
        st = wedge.wedge_run_bfs(G.handle, 0, out, o)
        np.testing.assert_array_equal(u32(out)[: g16.V], oracle.bfs_push(g16, 0))
        o = opts("sssp", switch=wedge.SWITCH_LEARNED)
        wedge.wedge_run_sssp(G.handle, 0, out, o)
        np.testing.assert_array_equal(u32(out)[: g16.V], oracle.sssp_dijkstra(g16, 0))
        assert st.iters > 0
    finally:
        G.close()
