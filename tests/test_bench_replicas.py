"""The multi-GPU form of bench.py is independent replicas (the invasion is
serial per image): no collective on the data path, only the job's time
reduced as the slowest rank's.  Checked here with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + 5 r ms per step and processed 1000 voxels
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        rate = bench.job_rate(1000, world, ms * 1e-3)
        # a second reduction in the same order on every rank
        e2e = bench.max_over_ranks(3.0 - rank, world, "cpu")
        out.put((rank, ms, rate, e2e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, e2e in res:
        assert ms == 15.0               # the slower rank's time
        assert rate == pytest.approx(2 * 1000 / 0.015)
        assert e2e == 3.0


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
