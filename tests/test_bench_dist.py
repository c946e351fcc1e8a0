"""The multi-rank timing path of bench.py with 2 gloo ranks on CPU: the job time is the
slowest rank's, and the whole-job value counts the units of every replica."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 40.0][rank]
    job = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (job, bench.replica_throughput(world, 1000, job))
    dist.destroy_process_group()


def test_two_rank_job_time_is_max_and_value_counts_all_replicas():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    job, value = res[0]
    assert job == 40.0
    assert value == pytest.approx(2 * 1000 / 0.040)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_throughput(1, 10, 2.0) == pytest.approx(5000.0)
