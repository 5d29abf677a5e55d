"""Multi-rank host logic of the benchmark, on CPU ranks (gloo): the job time
is the slowest rank's, and every rank gets the same value."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank, world, torch.device("cpu"), torch)
    dist.destroy_process_group()


def test_max_over_ranks_takes_the_slowest_rank():
    import bench
    assert bench.max_over_ranks(3.25, 1, None, torch) == 3.25
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert [out[r] for r in range(world)] == [2.5, 2.5]
