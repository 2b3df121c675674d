"""The multi-GPU form of the benchmark is replicas only (one independent
simulation per rank, no data-path collective): its host logic -- the job's
time as the maximum over the ranks after a barrier, the whole-job rate as
the ranks' units over that time -- checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group('gloo', init_method=f'tcp://127.0.0.1:{port}', rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = [12.5, 40.0][rank]  # rank 1 is the slow one
        t = bench.max_over_ranks(torch, dist, ms, 'cpu')
        out[rank] = (t, bench.job_rate(1000, world, t * 1e-3))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 40.0
    assert out[0][1] == pytest.approx(2 * 1000 / 0.040 / 1e6)


def test_single_rank_is_the_value_itself():
    assert bench.max_over_ranks(torch, None, 7.25, 'cpu') == 7.25
    assert bench.job_rate(5e6, 1, 2.0) == 2.5
