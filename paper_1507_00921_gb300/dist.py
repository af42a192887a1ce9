"""Multi-GPU partitioning for DBP: independent waveforms (and overlap-save blocks,
Section III) shard across ranks with no exchange on the data path.

One process per GPU (torchrun); each rank backpropagates its own waveforms.  The only
collectives are for measurement: the maximum elapsed time over ranks and the sum of
processed units.  Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def shard(n_items: int, world: int, rank: int):
    """Contiguous near-equal partition: returns (start, count) of this rank's items."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity without a group)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_over_ranks(values, device="cpu"):
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()


def throughput(units_per_rank: float, world: int, steps: int, seconds_max: float) -> float:
    """Whole-job rate: units of all ranks over the slowest rank's time (weak scaling)."""
    return units_per_rank * world * steps / seconds_max
