"""Replicas under torchrun (one process per GPU, no exchange on the data path): the
whole-job time is the slowest rank's and the work is summed over ranks.  Exercised
here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.replica_totals(10.0 + 3.0 * rank, 100.0 * (rank + 1), dist)
    dist.barrier()
    q.put((rank, ms, work))
    dist.destroy_process_group()


def test_replica_totals_take_max_time_and_summed_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 13.0, 300.0), (1, 13.0, 300.0)]


def test_single_gpu_is_the_identity():
    import bench
    assert bench.replica_totals(5.0, 7.0, None) == (5.0, 7.0)
