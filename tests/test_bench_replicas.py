"""The N > 1 path of bench.py (independent replicas, one per rank): the whole-job value counts
every rank's targets over the slowest rank's time. Two gloo ranks on CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [80.0, 125.0][rank]  # this rank's K-step time
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms, bench.replica_value(40000, world, 20, ms))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_whole_job_value():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        ms, value = out[r]
        assert ms == 125.0                                   # the slowest rank on every rank
        assert value == pytest.approx(40000 * 2 * 20 / 0.125)  # both ranks' targets


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.replica_value(1000, 1, 10, 5.0) == pytest.approx(2e6)
