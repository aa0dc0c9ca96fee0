"""Host logic of the learned switch's tooling: the fullness band learned from
traces (outside it one candidate was always the fastest) and the choice made
with it."""
import numpy as np

from paper_1903_07754_gb300 import costmodel


def _trace(xs, best):
    n = len(xs)
    feat = np.zeros((n, 6, 12), dtype=np.float32)
    feat[:, :, 2] = np.asarray(xs, dtype=np.float32)[:, None]
    ms = np.ones((n, 6))
    ms[np.arange(n), best] = 0.5
    return feat, ms, np.zeros(n, dtype=np.uint32)


def test_band_brackets_the_iterations_where_the_choice_varies():
    # fastest: k0 (1) at tiny fullness, k=2 (3) and dense (0) in between,
    # then k0 once more, dense (0) at large fullness
    tr = [_trace([1e-5, 2e-5, 0.01, 0.03, 0.2, 0.9], [1, 1, 3, 0, 1, 0]),
          _trace([5e-6, 0.05, 0.6], [1, 2, 0])]
    lo, hi = costmodel.learn_band(tr, pad=1.0)
    assert lo == np.float32(0.01)      # first fullness where k0 was clearly slower
    assert hi == np.float32(0.2)       # last fullness where dense was clearly slower
    lo2, hi2 = costmodel.learn_band(tr, pad=2.0)
    assert lo2 == lo / 2 and hi2 == hi * 2


def test_differences_within_noise_do_not_widen_the_band():
    feat, ms, ch = _trace([1e-5, 0.3], [1, 0])
    ms[0, 2] = 0.5 * 1.02   # k = 1 within 5% of k = 0 at the tiny frontier
    lo, hi = costmodel.learn_band([(feat, ms, ch)], pad=1.0)
    assert lo == np.float32(0.3) and hi == np.float32(1e-5) or hi <= lo


def test_band_of_one_sided_traces():
    # k0 always fastest: open below, dense nowhere fastest -> hi at the
    # largest fullness seen (padded); the model is needed in between
    lo, hi = costmodel.learn_band([_trace([1e-3, 1e-2], [1, 1])])
    assert lo == hi == np.float32(1e-2) * 2
    # dense always fastest: k0 clearly slower everywhere -> the model is
    # needed nowhere above half the smallest fullness seen
    lo, hi = costmodel.learn_band([_trace([0.3, 0.5], [0, 0])])
    assert lo == hi == np.float32(0.3) / 4


def test_choice_outside_the_band(monkeypatch):
    feat, _, _ = _trace([1e-4, 0.05, 0.7], [1, 1, 1])
    monkeypatch.setattr(costmodel, "choose", lambda params, f: np.full(f.shape[0], 4))
    got = costmodel.choose_in_band(None, feat, (1e-3, 0.5))
    np.testing.assert_array_equal(got, [1, 4, 0])
