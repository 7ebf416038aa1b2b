"""Query-sharded serving over graph replicas, one process per GPU.

Radial pattern queries are independent (Definition 1): every rank holds a
full copy of the knowledge graph on its own GPU and answers a share of the
queries; no collective touches the search itself.  The host side here deals
the queries round-robin, runs each rank's share through the library's
batched search and gathers the per-query results on one rank in the
original order (a host-side gather of small result records over
``torch.distributed``, gloo or NCCL).
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> list:
    """Query indices of `rank` among `world` ranks: round-robin, so uneven
    query costs spread evenly and every index belongs to exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return list(range(rank, n, world))


def search_sharded(kg, queries, group=None, dst: int = 0):
    """Run this rank's share of `queries` with ``kg.search_batch`` and gather
    every rank's (results, stats, status) triples on rank `dst`, in query
    order.  Returns the full list on `dst` and None on the other ranks.
    Without an initialised process group the call runs every query locally."""
    import torch.distributed as dist

    queries = list(queries)
    if not (dist.is_available() and dist.is_initialized()):
        return kg.search_batch(queries)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = shard(len(queries), rank, world)
    local = kg.search_batch([queries[i] for i in mine]) if mine else []
    parts = [None] * world if rank == dst else None
    dist.gather_object(list(zip(mine, local)), parts, dst=dst, group=group)
    if rank != dst:
        return None
    out = [None] * len(queries)
    for part in parts:
        for i, r in part:
            out[i] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"queries {missing[:8]} were answered by no rank")
    return out
