"""The benchmark's multi-process host logic, on CPU with two gloo ranks: every
rank agrees on the slowest rank's time (replicas run independently; the job
takes as long as the slowest one), and the reference arm runs on rank 0
only, the other ranks returning at once."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.reduce_max(10.0 * (rank + 1), world, torch.device("cpu"))
        ref = None
        if rank != 0:
            args = types.SimpleNamespace(scale=bench.SCALE, steps=3, warmup=1, ref_pr_iters=bench.PR_ITERS)
            ref = bench.run_reference(args, rank, world)
        dist.barrier()
        q.put((rank, got, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(got == pytest.approx(20.0) for _, got, _ in res)
    assert res[1][2] is None  # rank 1 does no reference work


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1, None) == 3.5
