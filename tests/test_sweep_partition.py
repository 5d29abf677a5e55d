"""Sharding of the batched sweep over ranks (host logic, gloo on CPU)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as wl
from paper_1905_05110_gb300.sweep import member_nodes, partition_members


def test_partition_is_complete_disjoint_and_balanced():
    nodes = member_nodes(wl.viv_sweep())
    for world in (1, 2, 3, 4, 8):
        parts = partition_members(nodes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(nodes)))
        loads = [sum(nodes[k] for k in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest member
        assert max(loads) - sum(loads) / world <= max(nodes)


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
    nodes = member_nodes(wl.viv_sweep())
    mine = partition_members(nodes, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out[rank] = gathered
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_ranks_agree_on_the_partition_without_exchanging_it(world):
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    views = [out[r] for r in range(world)]
    assert views[0] == views[1]
    flat = sorted(k for p in views[0] for k in p)
    assert flat == list(range(64))
    assert set(views[0][0]).isdisjoint(views[0][1])
