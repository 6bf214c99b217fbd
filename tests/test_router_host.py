"""Serving replicas across GPUs (ibip_route_pick, ibip.route_requests): the
routing rule on the host, and a request stream split over two gloo ranks
that agree on the split without exchanging anything, each rank serving its
share with a stand-in server (no GPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ibip():
    sys.path.insert(0, ROOT)
    from paper_2101_03240_gb300 import build_lib, ibip
    build_lib.build()
    return ibip


def test_route_pick_rule(ibip):
    assert ibip.route_pick([5, 3, 3, 9], [10] * 4, 1) == 1            # least load, lowest index on ties
    assert ibip.route_pick([5, 3, 3, 9], [10, 0, 10, 10], 1) == 2     # replica 1 cannot hold the job
    assert ibip.route_pick([0, 0], [4, 4], 5) == -1                   # nobody can
    assert ibip.route_pick([7], [1], 1) == 0
    with pytest.raises(ibip.IbipError):
        ibip.route_pick([1, 2], [3, 4], -1)


def test_route_requests_balances_greedily(ibip):
    vox = [100, 50, 50, 10, 200, 5, 5, 80]
    a = ibip.route_requests(vox, 3)
    # by hand: 100->0, 50->1, 50->2, 10->1 (50<=50, lowest), 200->2 (60 vs 50 -> replica 2 has 50)
    assert a[:5] == [0, 1, 2, 1, 2]
    loads = [sum(v for v, r in zip(vox, a) if r == k) for k in range(3)]
    assert max(loads) - min(loads) <= max(vox)
    assert ibip.route_requests(vox, 1) == [0] * len(vox)


class StubServer:
    """Stands in for ibip.Server on the host: records what it served."""

    def __init__(self):
        self.served = []

    def submit(self, j):
        self.served.append(j)
        return len(self.served) - 1

    def wait(self, t):
        return {"request": self.served[t], "status": 0}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, vox, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2101_03240_gb300 import ibip
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assign = ibip.route_requests(vox, world)
        srv = StubServer()
        tickets = [srv.submit(j) for j, r in enumerate(assign) if r == rank]
        done = [srv.wait(t)["request"] for t in tickets]
        everyone = [None] * world
        dist.all_gather_object(everyone, done)
        out.put((rank, assign, everyone))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_a_stream_without_messages(ibip):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2101_03240_gb300 import synth
    reqs = synth.c5_requests(n=120)
    vox = [L ** 3 for _, L, _ in reqs]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, vox, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a0, e0), (_, a1, e1) = res
    assert a0 == a1 == ibip.route_requests(vox, world)         # both ranks made the same split
    served = e0[0] + e0[1]
    assert sorted(served) == list(range(len(vox)))               # every request served exactly once
    loads = [sum(vox[j] for j in e0[k]) for k in range(world)]
    assert abs(loads[0] - loads[1]) <= max(vox)                 # balanced within one request
