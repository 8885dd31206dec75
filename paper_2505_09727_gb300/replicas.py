"""Coordination of one-process-per-GPU runs (torchrun, one rank per GPU).

A single system does not split across GPUs without a halo and transpose
exchange, so several GPUs run replicas: every rank solves its own copy of the
workload (or its own share of independent systems) and no data crosses ranks.
Only timings are combined: the job time is the slowest rank's (a MAX
all-reduce after a barrier), and the whole-job rate is the units all ranks
processed divided by that time.
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def init(backend: str) -> None:
    """Join the process group ("nccl" on GPUs, "gloo" on CPU) from env://."""
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend, init_method="env://")


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(values, device=None) -> list[float]:
    """Element-wise maximum of `values` over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / seconds


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous share of n_units for `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def finalize() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
