"""Data-parallel replicas: one process per GPU, one st_ctx per process.

Events are independent (each is reconstructed on its own, Section 2), so a job
is split into per-rank batches with no data exchange between ranks; results
stay with the rank that produced them.  The only collectives are on the host
side of the measurement: a barrier before timing and the maximum of the
ranks' elapsed times (the job ends when its slowest rank does).

Works with any torch.distributed backend: NCCL reduces a CUDA tensor, gloo a
CPU one.
"""

from __future__ import annotations

import os
from typing import Tuple


def dist_env() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return ws, rank, local


def shard(n_events: int, world_size: int, rank: int) -> Tuple[int, int]:
    """Contiguous event range [lo, hi) of `rank` when a fixed job of
    n_events is split over world_size ranks (sizes differ by at most one)."""
    if world_size < 1 or not 0 <= rank < world_size or n_events < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n_events, world_size)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def replica_seed(base: int, rank: int) -> int:
    """Generator seed of a rank's own batch (weak scaling: every rank
    processes a batch of the same size and statistics, different events)."""
    return base + rank


def _dist():
    try:
        import torch.distributed as dist
    except ImportError:  # pragma: no cover
        return None
    return dist if dist.is_available() and dist.is_initialized() else None


def barrier() -> None:
    d = _dist()
    if d is not None:
        d.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the value itself without a
    process group).  `device` is the CUDA device for NCCL; ignored by gloo."""
    d = _dist()
    if d is None:
        return float(value)
    import torch
    dev = device if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    if seconds <= 0:
        raise ValueError("non-positive time")
    return units_per_rank * world_size / seconds
