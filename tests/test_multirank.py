"""The bench's multi-rank host logic on two gloo ranks (CPU): the job time is
the slowest rank's, the throughput counts the units of every rank (weak
scaling, independent replicas, no data-path collective), and the reference
arm runs on rank 0 only."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        ms_local = 100.0 * (rank + 1)  # rank 1 is the slow one
        ms, value = bench.job_throughput(ms_local, units_per_rank=2e9, steps=5, world=world)
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # both ranks agree on the slowest rank's time
    assert res[0][0] == res[1][0] == 200.0
    # whole-job throughput: 2 ranks x 5 steps x 2e9 units in 0.2 s = 100 (x 1e9 units/s)
    assert res[0][1] == pytest.approx(100.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(250.0, 1e9, 4, 1) == (250.0, pytest.approx(16.0))


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        small = True
        steps = 1
        warmup = 0
        gpus = 2

    bench.run_reference(Args())  # returns at once on a non-zero rank
    assert capsys.readouterr().out == ""
