"""The replica aggregation of bench.py (independent copies of the workload,
one per rank, no data-path collective): whole-job rate = all ranks' node
updates / the slowest rank's time.  World size 2 over gloo on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [2.0, 3.0][rank]
    nodes = [100.0, 300.0][rank]
    rate, tmax = bench.aggregate(dist, secs, nodes, "cpu")
    out.put((rank, rate, tmax))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, rate, tmax in res:
        assert tmax == pytest.approx(3.0)
        assert rate == pytest.approx(400.0 / 3.0)


def test_aggregate_single_process():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, 2.0, 10.0) == (5.0, 2.0)
