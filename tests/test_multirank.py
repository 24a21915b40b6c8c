"""N > 1 ranks of bench.py on the CPU (gloo, world size 2): the replicas'
timings are combined as the slowest rank's and the job throughput counts
every rank's units (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    value, total = bench.job_throughput(local_ms, 1000.0, 3, world, dist)
    out[rank] = (value, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_all_units():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        value, total = out[r]
        assert total == 150.0
        assert abs(value - world * 1000.0 * 3 / 0.150) < 1e-6 * value


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, total = bench.job_throughput(200.0, 10.0, 4, 1, None)
    assert total == 200.0 and abs(value - 10.0 * 4 / 0.2) < 1e-9
