"""The multi-GPU path of bench.py is replicas (weak scaling): every rank
transforms its own seeded batch and the job's time is the max over ranks.
Its host logic runs here as two gloo processes on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank                 # ranks finish at different times
        ms = bench.job_ms(ms_local, world, dist, "cpu")
        value = bench.job_value(1000.0, world, 4, ms)
        out[rank] = (ms, value, bench.rank_seed(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_max_time_and_whole_job_value():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (ms0, v0, s0), (ms1, v1, s1) = out[0], out[1]
    assert ms0 == ms1 == 15.0                        # the slowest rank sets the job time
    assert v0 == v1 == pytest.approx(1000.0 * 2 * 4 / 15e-3)
    assert s0 != s1                                  # each rank its own batch


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A(), 1) is None       # rank 1: no work, nothing printed
    assert capsys.readouterr().out == ""
