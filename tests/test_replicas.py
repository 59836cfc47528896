"""The multi-GPU form of bench.py: N independent replicas, one per rank, whose
whole-job rate is every rank's work over the slowest rank's time.  The
aggregation runs here on CPU ranks with the gloo backend (world size 2)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 5.0][rank]          # the second rank is the slow one
    evals = [100, 100][rank]
    rate, slowest = bench.replica_rate(seconds, evals, 10.0, dist, "cpu")
    out.put((rank, rate, slowest))
    dist.destroy_process_group()


def test_replica_rate_uses_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slowest in res:
        assert slowest == 5.0               # max over ranks, seen by every rank
        assert rate == 2 * 100 * 10.0 / 5.0  # all ranks' work over the slowest time


def test_replica_rate_single_process():
    import bench
    assert bench.replica_rate(4.0, 50, 2.0) == (25.0, 4.0)
