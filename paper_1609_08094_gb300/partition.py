"""Partition of the task list (sorted occupied triples, Sec. 3) across ranks.

Tasks are independent and of equal weight (Sec. 5), so one process per GPU
takes a contiguous range of the list and the only exchange is the final sum
of three numbers -- no collective on the data path.
"""
from __future__ import annotations


def rank_range(ntask: int, rank: int, world: int):
    """(first, count) of rank's share of a whole job: contiguous, sizes
    differing by at most one."""
    if world < 1 or not 0 <= rank < world or ntask < 0:
        raise ValueError("bad rank/world/ntask")
    base, extra = divmod(ntask, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def step_batch(ntask: int, rank: int, world: int, step: int, count: int):
    """First task of rank's batch of ``count`` tasks at ``step`` of a
    weak-scaling run: the ranks' batches of one step are disjoint, and
    successive steps move through the list (wrapping around)."""
    if count < 1 or count > ntask:
        raise ValueError("count must be in [1, ntask]")
    span = ntask - count + 1  # valid first indices
    return ((step * world + rank) * count) % span
