"""Multi-GPU layout of the V_loc action: bands shard across ranks.

Bands are independent, so a block of nbands is split into contiguous
per-rank shards; every rank holds the plan and V.  The forward and adjoint
applies need no collective.  The backward's dL/dV is a sum over bands, so
the per-rank partial sums are added with one all-reduce of N reals.  Timing
across ranks takes the maximum (the slowest rank sets the step time).
These helpers only move rank-level scalars and the dV sum; every band's
arithmetic runs in the CUDA kernels on its own rank.
"""
from __future__ import annotations


def band_shard(nbands: int, rank: int, world: int) -> tuple[int, int]:
    """(first band, count) of `rank`'s contiguous shard of nbands bands."""
    if world < 1 or not 0 <= rank < world or nbands < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(nbands, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_grad_v(grad_v):
    """Sum the per-rank partial dL/dV (in place) over the default group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(grad_v, op=dist.ReduceOp.SUM)
    return grad_v


def aggregate_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: units over all ranks / the slowest rank's time."""
    return units_per_rank * world / seconds_max
