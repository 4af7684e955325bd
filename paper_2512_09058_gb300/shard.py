"""Host-side logic of multi-GPU runs over independent OCPs (weak scaling).

Every rank solves its own batch: rank r takes instances r*n .. (r+1)*n-1 of a
workload (each instance is drawn from its own seed stream, so a rank's shard
is the same whatever the world size).  There is no data-path collective; the
only cross-rank step is the reduction of the step time (the slowest rank
defines the job's time) and the sum of the work."""
from __future__ import annotations


def shard_indices(n_per_rank: int, rank: int):
    return range(rank * n_per_rank, (rank + 1) * n_per_rank)


def reduce_time_ms(ms: float, dist=None, device=None) -> float:
    """Maximum over ranks of a per-rank time (no-op without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)
