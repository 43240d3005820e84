"""The bench's multi-GPU mode is replicas only: each rank transforms its own
image and the job's time is the slowest rank's. Its host-side logic runs here
as two gloo ranks on the CPU."""

import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import edges_and_lines
    local_ms = [12.5, 20.0][rank]
    total = bench.reduce_max_ms(local_ms, world, torch.device("cpu"))
    img = edges_and_lines(64, 64, seed=4096 + rank)
    dist.barrier()
    results[rank] = (total, bench.whole_job_mpix_s(world, 4096 * 4096, total / 10),
                     int(img.sum()), img.tobytes().__hash__())
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert res[0][0] == res[1][0] == 20.0
    assert np.isclose(res[0][1], 2 * 4096 * 4096 / 1e6 / (2.0 / 1e3))
    assert res[0][3] != res[1][3]       # each rank its own image
