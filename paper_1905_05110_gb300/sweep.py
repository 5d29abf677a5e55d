"""Host logic of the batched parameter sweep across ranks.

A sweep is many independent simulations (uneven lattices); it shards across
GPUs with no exchange step: every rank computes the same deterministic
partition and runs its members in one batch.  Only the end of the run meets
(timing, optional gather of the histories).
"""
from __future__ import annotations


def partition_members(node_counts, world_size: int):
    """Greedy longest-processing-time split of members over ranks.

    Members are taken by decreasing node count (ties by index) and each goes
    to the rank with the fewest nodes so far (ties to the lowest rank).  The
    result is the same on every rank.  Returns a list of sorted member-index
    lists, one per rank.
    """
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(node_counts)), key=lambda k: (-int(node_counts[k]), k))
    loads = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for k in order:
        r = min(range(world_size), key=lambda q: (loads[q], q))
        parts[r].append(k)
        loads[r] += int(node_counts[k])
    return [sorted(p) for p in parts]


def member_nodes(problems):
    return [int(p["nx"]) * int(p["ny"]) for p in problems]
