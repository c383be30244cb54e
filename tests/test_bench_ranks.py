"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
gets the slowest rank's time, and the whole-job value counts the units of
all ranks over that time (replicas, weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [120.0, 250.0][rank]
    m = bench.reduce_max_ms(local, world, "cpu")
    v = bench.job_value(512 * 10, world, m)
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(f"{m} {v}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_and_job_value(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        m, v = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert m == 250.0
        assert abs(v - 512 * 10 * 2 / 0.25) < 1e-9


def test_single_rank_is_local_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_ms(3.5, 1, "cpu") == 3.5
    assert bench.job_value(100, 1, 1000.0) == 100.0
