"""Independent replicas across ranks.

The synapse search of one network does not shard in this library (it runs on
one GPU); several GPUs run independent networks.  The only cross-rank work is
host-side bookkeeping of the benchmark: a barrier before and after the timed
region and the slowest rank's time.  Works with any torch.distributed backend
(nccl on GPUs, gloo on CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def barrier() -> None:
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (e.g. the slowest rank's step time)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_throughput(units_this_rank: int, ms_this_rank: float, device=None) -> dict:
    """Whole-job throughput of independent replicas: all units over the slowest
    rank's time."""
    units = sum_over_ranks(units_this_rank, device)
    ms = max_over_ranks(ms_this_rank, device)
    return {"units": int(units), "ms": ms, "per_s": units / (ms / 1e3) if ms > 0 else 0.0}
