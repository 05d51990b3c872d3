"""The N>1 path of bench.py on CPU ranks (gloo, world size 2): every rank
works on its own seeded share with no data-path collective; the job time is
the max over ranks and the job rate counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own (seeded) share: different inputs per rank
        basis, batches = bench.sweep(seed=rank, only=(1, 0, 1, 0), nq=64)
        q = batches[(1, 0, 1, 0)][2]
        my_ms = 100.0 + 50.0 * rank
        mx = bench.reduce_max(my_ms, dist, torch.device("cpu"))
        out[rank] = (mx, float(q.sum()), bench.job_rate(world, 64, 3, mx))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_job_rate():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] != out[1][1]                      # ranks drew different seeded shares
    assert out[0][2] == pytest.approx(2 * 64 * 3 / 0.150)
