"""Replica bookkeeping for multi-GPU runs.

The density-matrix path has no data exchange: with N GPUs every rank evolves its own states (an
independent replica of the workload, or its share of a batch's instances). The only cross-rank
steps are a barrier around the timed region, the maximum of the per-rank times, and the sum of
the units of work. Those steps work with the ``gloo`` backend (CPU tensors) and with ``nccl``.
"""
from __future__ import annotations

import os
from typing import Sequence, Tuple

import torch
import torch.distributed as dist


def env() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment; (0, 1, 0) without it."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _device() -> torch.device:
    if dist.is_initialized() and dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def barrier() -> None:
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float) -> float:
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items: Sequence, rank: int, world: int) -> list:
    """Round-robin share of independent work items (batch instances) for one rank."""
    return [items[i] for i in range(rank, len(items), world)]


def job_throughput(units_per_rank: float, seconds_per_rank: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum_over_ranks(units_per_rank) / max_over_ranks(seconds_per_rank)
