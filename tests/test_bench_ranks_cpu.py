"""bench.py's whole-job rate over ranks (replicas only: each rank an independent
rollout, no collective on the data path): two gloo ranks on the CPU, each with its
own timed duration, must both report the slowest rank's time and the rate of all
ranks' steps over it; a single rank reports its own."""
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


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        elapsed, value = bench.whole_job_rate([2.0, 5.0][rank], 300, world, torch.device("cpu"))
        out[rank] = (elapsed, value)
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        assert res[r] == (5.0, 2 * 300 / 5.0)


def test_whole_job_rate_single_rank():
    assert bench.whole_job_rate(4.0, 200, 1, None) == (4.0, 50.0)
