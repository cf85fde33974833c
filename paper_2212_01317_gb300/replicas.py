"""Splitting one job across processes, one GPU each.

The method's units are independent (Sec. 2.1): every realization is its own
chain from the same start, differing only in its random numbers, and every
field (time slice) is its own problem. Two partitions follow.

* ``fields`` (weak scaling): each rank fills its own field with its own seed
  and slice id. No data-path collective; the job's time is the maximum over
  ranks and its work the sum.
* ``realizations`` (strong scaling over one field): rank 0 calibrates and
  broadcasts the n_blk block temperatures; every rank runs a disjoint range of
  realization indices; the per-site sums of the final states and their counts
  are added with one all-reduce of H*W doubles, after which every rank holds
  the job's accumulator and predicts the same field.

The collectives use whatever process group torch.distributed holds: NCCL on
device tensors on the GPU, gloo on host tensors in the CPU tests. Nothing
here computes any part of the method.
"""
from __future__ import annotations

import numpy as np


def shard_realizations(R: int, world: int, rank: int) -> tuple[int, int]:
    """First realization index and count of `rank`: [0, R) cut into `world`
    contiguous ranges whose sizes differ by at most one."""
    if R < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("need R >= 0, world >= 1, 0 <= rank < world")
    base, extra = divmod(R, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int, mode: str) -> tuple[int, int]:
    """(seed, slice id) of a rank. Fields mode: every rank a different field,
    so a different seed and slice id. Realizations mode: one field, so the
    same seed and slice id; the realization index separates the streams."""
    if mode == "fields":
        return (seed + 7919 * rank) & (2**64 - 1), rank
    if mode == "realizations":
        return seed, 0
    raise ValueError(f"unknown mode {mode}")


def _dist():
    import torch.distributed as dist
    return dist


def max_over_ranks(value: float, device=None) -> float:
    """The job's time: the slowest rank's."""
    import torch
    dist = _dist()
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """The job's work: the sum of every rank's."""
    import torch
    dist = _dist()
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def broadcast_temperatures(T, src: int = 0):
    """Rank `src`'s block temperatures to every rank, in place (a float32 tensor)."""
    dist = _dist()
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.broadcast(T, src=src)
    return T


def allreduce_accumulator(acc, count: int) -> int:
    """Adds every rank's per-site sums (a float64 tensor, in place) and returns
    the total number of realizations they hold."""
    import torch
    dist = _dist()
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return int(count)
    dist.all_reduce(acc)
    n = torch.tensor([int(count)], dtype=torch.int64, device=acc.device)
    dist.all_reduce(n)
    return int(n.item())


def fill_shared_field(ctx, R: int, world: int, rank: int, acc, T):
    """Realizations mode through the C-ABI: `ctx` is this rank's context of
    the shared field, `acc` a float64 device tensor of H*W elements, `T` a
    float32 device tensor of n_blk elements. Rank 0 calibrates, every rank
    runs its share of the R realizations, the sums are added, and `ctx` ends
    up holding the job's accumulator (ready for mpr_predict)."""
    from . import mpr
    if rank == 0:
        mpr.mpr_calibrate(ctx, T)
    broadcast_temperatures(T, 0)
    if rank != 0:
        mpr.mpr_set_temperatures(ctx, T)
    first, count = shard_realizations(R, world, rank)
    mpr.mpr_set_realization_base(ctx, first)
    if count > 0:
        mpr.mpr_simulate(ctx, count)
    n = mpr.mpr_get_accumulator(ctx, acc)
    total = allreduce_accumulator(acc, n)
    mpr.mpr_set_accumulator(ctx, acc, total)
    return first, count, total


def check_partition(R: int, world: int) -> np.ndarray:
    """Every realization index covered exactly once (for tests and asserts)."""
    seen = np.zeros(R, np.int64)
    for r in range(world):
        f, c = shard_realizations(R, world, r)
        seen[f:f + c] += 1
    return seen
