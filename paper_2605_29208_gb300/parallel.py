"""Data-parallel Baum-Welch across processes (one GPU each).

The E-step shards sequences across ranks with no communication; the one
exchange of an iteration is the element-wise sum of the float64 statistic
records (every entry is a sum over sequences), after which every rank runs
the same M-step and holds identical models.
"""
from __future__ import annotations


def shard(n_seq: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of sequences [lo, hi) owned by `rank`."""
    base, extra = divmod(n_seq, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_stats(record, group=None):
    """Sums a statistic record tensor over all ranks in place (NCCL for CUDA
    tensors, gloo for CPU tensors)."""
    import torch.distributed as dist
    dist.all_reduce(record, op=dist.ReduceOp.SUM, group=group)
    return record
