"""Data-parallel replicas: one process per GPU, each evaluating its own
queries (geometry pairs are independent, so there is no exchange on the data
path).  Only the timing is combined: every rank's timed region is bracketed
by a barrier and the job's time is the maximum over ranks.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str):
    """Initialise the default process group when WORLD_SIZE > 1; returns the
    torch.distributed module, or None for a single process."""
    ws, _, _ = env()
    if ws <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(value: float, dist, device="cpu") -> float:
    """The largest `value` of all ranks (the job's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world_size: int, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest
    rank's time (weak scaling: every rank processes units_per_rank)."""
    return units_per_rank * world_size / (max_ms / 1000.0)
