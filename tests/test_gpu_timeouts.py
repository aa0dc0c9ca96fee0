"""Failure detection without a GPU fault: every device wait in the library is
bounded, gives up after 200 ms and reports WEDGE_ERR_TIMEOUT to the host.  A
wait that nothing can satisfy (an mbarrier missing an arrival, a grid
barrier that one block never reaches) must come back with that status, and
the device must stay usable for the next run."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from _gpu import empty_u32, graph, u32
from paper_1903_07754_gb300 import wedge

pytestmark = pytest.mark.gpu

TIMEOUT = 4


@pytest.mark.parametrize("kind", [0, 1])
def test_unsatisfiable_wait_times_out_and_device_recovers(kind):
    t0 = time.time()
    assert wedge.wedge_selftest_timeout(kind) == TIMEOUT
    assert time.time() - t0 < 30
    g = gg.rmat(10, 8, seed=3)
    G = graph(g, with_weights=False)
    try:
        out = empty_u32(g.V)
        wedge.wedge_run_bfs(G.handle, 0, out)
        np.testing.assert_array_equal(u32(out)[: g.V], oracle.bfs_push(g, 0))
    finally:
        G.close()


def test_selftest_rejects_unknown_kind():
    assert wedge.wedge_selftest_timeout(7) == 1
