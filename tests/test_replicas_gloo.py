"""The multi-GPU benchmark path runs independent replicas: each rank answers
its own queries and the job time is the slowest rank's.  Checked here with two
gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    my_ms = 100.0 + 50.0 * rank            # rank 1 is the slow replica
    total = bench.max_over_ranks(my_ms, dist, device="cpu")
    out[rank] = bench.job_throughput(total, steps=10, world=world)
    dist.destroy_process_group()


def test_two_replicas_report_job_throughput_over_the_slowest_rank():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    # 2 ranks x 10 queries over the slowest rank's 150 ms
    assert out[0] == out[1] == world * 10 / 0.150


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(500.0, steps=10, world=1) == 20.0
