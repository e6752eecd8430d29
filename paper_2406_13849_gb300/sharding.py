"""Spreading the tracking work over several GPUs (one process per GPU).

Histories are independent and every random number is keyed by the particle
id, so a run split into contiguous id ranges, one per rank, computes exactly
the histories of the unsplit run (the paper's replicated-domain runs: every
rank holds the whole geometry).  The only exchange is the merge of the
tallies and counters at the end: integer sums, so the merged result does not
depend on the split or on the order of the reduction.  A batch of many
geometries is split by geometry instead (each rank runs whole problems).

The reduction uses torch.distributed (NCCL between GPUs, gloo on CPU ranks);
these helpers only choose the ranges and issue the collectives.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

# counters[STATUS] holds the first kernel-level status (0 = none, negative
# codes); it is merged by MIN so that any rank's failure survives
STATUS = 15


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first particle id, count) of rank's contiguous share of n_total ids;
    the first n_total % world ranks take one more."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("shard_range: bad rank/world/n_total")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def merge_tallies(tally: torch.Tensor, counters: torch.Tensor | None = None, group=None) -> None:
    """In place: the sum over ranks of the uint64 tallies (stored in int64
    tensors; two's-complement sums are the uint64 sums) and of the counters,
    except the status slot, merged by MIN."""
    if tally.dtype != torch.int64 or (counters is not None and counters.dtype != torch.int64):
        raise TypeError("merge_tallies: tallies and counters are int64 tensors")
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    if counters is not None:
        status = counters[STATUS:STATUS + 1].clone()
        counters[STATUS] = 0
        dist.all_reduce(counters, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(status, op=dist.ReduceOp.MIN, group=group)
        counters[STATUS] = status[0]


def shard_geometries(counts, world: int) -> list[list[int]]:
    """Indices of the geometries each rank runs: the largest populations
    first, each to the rank with the fewest particles so far (ties to the
    lower rank), so the ranks' loads differ by at most one geometry's."""
    loads = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(counts)), key=lambda i: (-int(counts[i]), i)):
        r = min(range(world), key=lambda j: (loads[j], j))
        out[r].append(k)
        loads[r] += int(counts[k])
    for lst in out:
        lst.sort()
    return out
