"""The multi-rank timing of bench.py (replicas only): two gloo ranks on CPU.

Each rank runs independent solves; the job's throughput is the solves summed
over ranks divided by the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, seconds = (10, 2.0) if rank == 0 else (12, 3.0)
    rate, total, tmax = bench.aggregate(units, seconds)
    out[rank] = (rate, total, tmax)
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        rate, total, tmax = res[r]
        assert total == 22.0 and tmax == 3.0 and abs(rate - 22.0 / 3.0) < 1e-12


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(5, 2.0) == (2.5, 5, 2.0)
