"""Multi-GPU use without a data-path collective: independent replicas.

The solves of different right-hand sides share nothing, so N GPUs run N
independent replicas (one process per GPU).  Rank r takes its own seeds; the
only collective is the max-reduction of the timed region that turns the
per-rank times into the job's time (the slowest rank bounds the job)."""
from __future__ import annotations


def seeds_for_rank(rank: int, world: int, per_rank: int) -> list[int]:
    """Disjoint seed ranges: rank r solves seeds r*per_rank .. (r+1)*per_rank-1."""
    if not 0 <= rank < world or per_rank < 0:
        raise ValueError("bad rank/world/per_rank")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def job_time(local_ms: float, world: int, device=None) -> float:
    """Max over ranks of the local timed region (identity for one process)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, world: int, job_ms: float) -> float:
    """Whole-job throughput: units of all ranks over the job's time."""
    return world * units_per_rank / (job_ms * 1e-3)
