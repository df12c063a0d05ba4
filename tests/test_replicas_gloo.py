"""The N > 1 path of bench.py runs one independent replica per rank (no data-
path collective) and reports the units of all ranks over the slowest rank's
time.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 * (rank + 1)                # rank 1 is the slowest: 20 ms
        dist.barrier()
        value, ms_max = bench.replica_throughput(ms, 1000 * 5, world, dist, "cpu")
        out[rank] = (value, ms_max)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, ms_max = res[r]
        assert ms_max == 20.0                 # max over ranks, seen by every rank
        assert value == pytest.approx(2 * 1000 * 5 / 0.020)


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    value, ms_max = bench.replica_throughput(8.0, 400, 1)
    assert ms_max == 8.0 and value == pytest.approx(400 / 0.008)
