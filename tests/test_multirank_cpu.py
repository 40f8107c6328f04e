"""The multi-rank path of bench.py on CPU: two gloo ranks, each an independent replica,
reported as whole-job throughput over the slowest rank's time (no data-path collective)."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [1000.0, 1500.0][rank]
    value, total = bench.aggregate(world, coeffs_per_step=4, steps=3, total_ms=local_ms, device="cpu")
    out[rank] = (value, total)
    assert bench.dist_env()[:2] == (rank, world)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, total = out[r]
        assert total == 1500.0                    # max over ranks
        assert value == pytest.approx(2 * 4 * 3 / 1.5)  # every rank's coefficients over the slowest time


def test_single_rank_has_no_collective():
    import bench

    value, total = bench.aggregate(1, coeffs_per_step=10, steps=2, total_ms=500.0, device="cpu")
    assert (value, total) == (40.0, 500.0)
