"""Sharding of independent work units across ranks (one process per GPU).

Amplitudes of different bitstrings, prefix groups and slices are independent,
so ranks never exchange data on the contraction path: each rank takes a
contiguous share of the units, and only the timing of a benchmark is reduced
(max over ranks).  The only data reduction the method has, the FP64 sum of a
sliced amplitude over its slices, is `allreduce_sum_c128`.
"""
from __future__ import annotations

import numpy as np

from rqc_inputs import prefix_group_bitstrings


def shard(n_units: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's contiguous share of n_units (sizes differ by at
    most one, lower ranks take the larger shares)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def rank_prefix_batch(R: int, C: int, prefix_cols: int, groups_per_rank: int, per_group: int,
                      seed: int, world: int, rank: int) -> np.ndarray:
    """This rank's bitstrings when every rank processes `groups_per_rank`
    prefix groups of a global batch of world * groups_per_rank groups (weak
    scaling: the per-rank work is fixed; rank 0 of a one-rank job gets the
    single-GPU batch)."""
    allbits = prefix_group_bitstrings(R, C, prefix_cols, world * groups_per_rank, per_group,
                                      seed)
    g0, g1 = shard(world * groups_per_rank, world, rank)
    return allbits[g0 * per_group:g1 * per_group]


def rank_slice_ids(ids, lower_mask: int, world: int, rank: int) -> list:
    """This rank's share of one amplitude's slices: whole runs of slices that
    share the odd-side lower half's bits (so that each rank keeps the lower
    half's reuse), the runs split contiguously over the ranks.  Each rank sums
    its slices; allreduce_sum_c128 adds the ranks' partial amplitudes."""
    runs = {}
    for i in sorted(int(v) for v in ids):
        runs.setdefault(i & lower_mask, []).append(i)
    keys = sorted(runs)
    g0, g1 = shard(len(keys), world, rank)
    return [i for k in keys[g0:g1] for i in runs[k]]


def max_over_ranks(value: float, dist, device=None) -> float:
    """Max of a float over all ranks (the timing rule of the benchmark)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum_c128(a: np.ndarray, dist, device=None) -> np.ndarray:
    """Sum of complex128 partial amplitudes over ranks (slices spread across
    ranks), in FP64."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy().view(np.complex128)
