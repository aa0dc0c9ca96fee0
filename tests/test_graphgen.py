"""Checks of the seeded input generators (shared inputs, not the method)."""
import numpy as np

import graphgen as gg


def _check_csc(g):
    off = g.offsets.astype(np.int64)
    assert off[0] == 0 and off[-1] == g.E and np.all(np.diff(off) >= 0)
    dst = g.dst().astype(np.int64)
    src = g.src.astype(np.int64)
    key = dst * g.V + src
    assert np.all(np.diff(key) > 0)          # sorted by (dst, src), no duplicates
    assert not np.any(src == dst)            # no self-loops


def test_rmat_layout_and_determinism():
    a = gg.rmat(12, 16)
    b = gg.rmat(12, 16)
    _check_csc(a)
    np.testing.assert_array_equal(a.src, b.src)
    assert a.E < 16 << 12


def test_rmat_quadrant_frequencies():
    """Top-level quadrant shares of the raw samples approach a, b, c, d."""
    g = gg.rmat(14, 16, seed=11)
    src, dst = g.src.astype(np.int64), g.dst().astype(np.int64)
    top = 1 << 13
    q = (src >= top) * 2 + (dst >= top)
    share = np.bincount(q, minlength=4) / q.size
    # deduplication removes mostly quadrant-0 repeats, so allow a margin
    assert share[0] > 0.45 and share[3] < 0.1
    assert abs(share[1] - share[2]) < 0.01


def test_grid_structure():
    g = gg.grid(16, 0.0)
    _check_csc(g)
    assert g.E == 2 * 2 * 16 * 15
    deg = g.indeg()
    assert deg.max() == 4 and deg.min() == 2
    r = gg.grid(64, 0.01)
    _check_csc(r)
    np.testing.assert_array_equal(r.indeg(), r.outdeg())  # undirected


def test_symmetrize_and_weights():
    g = gg.rmat(10, 8)
    s = gg.symmetrize(g)
    _check_csc(s)
    np.testing.assert_array_equal(s.indeg(), s.outdeg())
    w = g.with_weights(255).w
    assert w.min() >= 1 and w.max() <= 255
    assert gg.weight(3, 7, 2, 255) == gg.weight(3, 7, 2, 255)


def test_roots_have_out_edges():
    g = gg.rmat(12, 4)
    r = gg.roots(g, 64)
    assert np.all(g.outdeg()[r] > 0)
    np.testing.assert_array_equal(r, gg.roots(g, 64))
