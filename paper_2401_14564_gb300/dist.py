"""Multi-process helpers for the data-parallel path (one process per GPU).

The method has no exchange between pixels or molecules, so ranks only split
work and agree on timings: `shard` gives each rank a contiguous share of n
independent units (molecules of a batch, pixel rows of a scan), and
`max_over_ranks` / `sum_over_ranks` reduce a host scalar with whatever
process group is initialised (NCCL on GPUs, gloo on CPU).  Without an
initialised group they return their input.
"""
from __future__ import annotations

import torch


def shard(n: int, rank: int, world: int):
    """Contiguous [start, stop) of n units for `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("invalid shard request")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _reduce(x: float, op, device=None) -> float:
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    import torch.distributed as dist

    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device=None) -> float:
    import torch.distributed as dist

    return _reduce(x, dist.ReduceOp.SUM, device)
