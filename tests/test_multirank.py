"""The N > 1 bench path on CPU: two gloo ranks reduce their times (max) and
units (sum) the way bench.py does on N GPUs, and replicas draw different
sources on the same graph. No GPU."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + rank, world, "cpu")
        edges = bench.sum_over_ranks(100.0 * (rank + 1), world, "cpu")
        dist.barrier()
        q.put((rank, ms, edges, bench.whole_job_gteps(edges, 3, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_available() or not torch.distributed.is_gloo_available():
        pytest.skip("gloo not available")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, edges, gteps in out:
        assert ms == 11.0  # the slowest rank's time
        assert edges == 300.0  # both ranks' units
        assert gteps == pytest.approx(300.0 * 3 / 11e-3 / 1e9)


def test_single_rank_reductions_are_identity():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(5.0, 1, "cpu") == 5.0
    assert bench.sum_over_ranks(7.0, 1, "cpu") == 7.0


def test_replicas_share_the_graph_and_draw_their_own_sources():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    a = bench.make_workload(10, 8, rank=0)
    b = bench.make_workload(10, 8, rank=1)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst) and np.array_equal(a.w, b.w)
    assert not np.array_equal(a.sources, b.sources)
