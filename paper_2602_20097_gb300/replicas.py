"""Replica helpers for running the method on several GPUs of one node.

The exact EDT does not shard with halos (a nearest boundary can be anywhere in
the field), so a multi-GPU job runs independent replicas: each rank mitigates
its own fields, and ranks only agree on timing. There is no collective on the
data path; :func:`max_over_ranks` is the one reduction, on the step time.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank ``rank``'s synthetic field (distinct per rank)."""
    return int(base) + int(rank)


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of ``n_items`` owned by ``rank`` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(n_items), int(world))
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Largest ``value`` over all ranks of the default process group (the
    value itself without one)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_rank: float, world: int, ms_max: float) -> float:
    """Aggregate throughput: the bytes all ranks processed over the slowest
    rank's time."""
    return float(bytes_per_rank) * int(world) / (float(ms_max) * 1e-3) / 1e9
