"""Multi-GPU runs are independent replicas: one process per GPU, each decoding
its own shot range, no collective on the data path.  These helpers hold the
host-side logic (shot ranges, the max-over-ranks time, the whole-job rate)
so it can be tested with the gloo backend on CPU.
"""
from __future__ import annotations


def shot_offset(rank: int, shots_per_rank: int) -> int:
    """First shot of a rank's range: ranks decode disjoint, equal-size ranges."""
    if rank < 0 or shots_per_rank < 0:
        raise ValueError("rank and shots_per_rank must be >= 0")
    return rank * shots_per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The slowest rank's time (the job finishes when the last replica does)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    if seconds <= 0:
        raise ValueError("seconds must be > 0")
    return units_per_rank * world / seconds
