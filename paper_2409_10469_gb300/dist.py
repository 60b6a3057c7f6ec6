"""Multi-process helpers of the benchmark: one process per GPU, each running its
own independent controller instance (MPPI instances share nothing, so there is
no data-path collective).  The only communication is the timing protocol:
a barrier before and after the timed region and the maximum step time over
ranks, from which the whole-job throughput is formed (weak scaling)."""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world_size: int, max_seconds: float) -> float:
    """Whole-job throughput under weak scaling: every rank processed
    units_per_rank; the job took the slowest rank's time."""
    return units_per_rank * world_size / max_seconds
