"""Host-side logic of running the path on several GPUs of one node: replicas, one process per GPU.

Events are independent (the paper's method has no cross-event state), so the work shards by event
with no collective on the data path: rank r of N takes its own events, and the only collectives
are the barrier around the timed region and the maximum of the ranks' times, from which the
whole-job throughput is formed (weak scaling: per-GPU work fixed as N grows).
"""
from __future__ import annotations


def event_indices(rank: int, world: int, per_rank: int, base: int = 0) -> list[int]:
    """Seeded event indices of one rank: a contiguous block, disjoint across ranks."""
    if world < 1 or not 0 <= rank < world or per_rank < 0:
        raise ValueError("need 0 <= rank < world and per_rank >= 0")
    start = base + rank * per_rank
    return list(range(start, start + per_rank))


def max_over_ranks(dist, value: float, device=None) -> float:
    """Largest `value` over the process group (the value itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("the timed region must have positive duration")
    return units_per_rank * world / max_seconds


def backend_for(cuda_available: bool) -> str:
    """NCCL between GPUs; gloo for the CPU-only runs that test this logic."""
    return "nccl" if cuda_available else "gloo"
