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
    # best: sparse k0 (1) at tiny fullness, k=2 (3) and dense (0) in between,
    # dense (0) at large fullness
    tr = [_trace([1e-5, 2e-5, 0.01, 0.03, 0.2, 0.9], [1, 1, 3, 0, 1, 0]),
          _trace([5e-6, 0.05, 0.6], [1, 2, 0])]
    lo, hi = costmodel.learn_band(tr, pad=1.0)
    assert lo == np.float32(0.01)      # first fullness whose best is not sparse k0
    assert hi == np.float32(0.2)       # last fullness whose best is not dense
    lo2, hi2 = costmodel.learn_band(tr, pad=2.0)
    assert lo2 == lo / 2 and hi2 == hi * 2


def test_band_of_one_sided_traces():
    # always sparse k0: nothing below needs the model (lo = 0), and above the
    # largest such fullness (padded) the traces say nothing -- dense
    lo, hi = costmodel.learn_band([_trace([1e-3, 1e-2], [1, 1])])
    assert lo == 0.0 and hi == np.float32(1e-2) * 2
    # always dense: the band starts at half the smallest fullness seen and is open above
    lo, hi = costmodel.learn_band([_trace([0.3, 0.5], [0, 0])])
    assert lo == np.float32(0.3) / 2 and hi == costmodel.NO_BAND[1]


def test_choice_outside_the_band(monkeypatch):
    feat, _, _ = _trace([1e-4, 0.05, 0.7], [1, 1, 1])
    monkeypatch.setattr(costmodel, "choose", lambda params, f: np.full(f.shape[0], 4))
    got = costmodel.choose_in_band(None, feat, (1e-3, 0.5))
    np.testing.assert_array_equal(got, [1, 4, 0])
