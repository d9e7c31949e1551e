"""Multi-GPU sharding of independent work units (one process per GPU).

Chunks of different streams are independent in the plain method (no temporal context), so the units are
sharded by stream: stream s runs on rank s mod world.  There is no data-path collective; the only
cross-rank traffic is the benchmark's barrier and the reduction of its timing (the slowest rank's span)
and of the units each rank processed.
"""
from __future__ import annotations


def shard(stream_ids, rank: int, world: int) -> list:
    """The streams rank `rank` of `world` owns: stream s -> rank s mod world (stream affinity)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    return [s for s in stream_ids if s % world == rank]


def aggregate(local_units: float, local_ms: float, dist=None, device=None) -> tuple[float, float]:
    """Whole-job throughput over ranks: (units of all ranks, the slowest rank's milliseconds).  value =
    units / (ms / 1000).  Without an initialised process group this is the local pair."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_units), float(local_ms)
    import torch
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
