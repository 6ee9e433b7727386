"""Multi-process helpers for the data-parallel path (one process per GPU).

The method has no exchange between pixels or molecules, so ranks only split
work and agree on timings: `shard` gives each rank a contiguous share of n
independent units (molecules of a batch, pixel rows of a scan), and
`max_over_ranks` / `sum_over_ranks` reduce a host scalar with whatever
process group is initialised (NCCL on GPUs, gloo on CPU).  Without an
initialised group they return their input.

The one exchange a single large system needs is in the backward: the loss
sum(w * df) is a sum over pixels, so when the ranks split the scan by pixel
rows, each rank's gradient of its own rows' terms adds up to the whole
image's gradient.  `reduce_grads` sums those per-atom and tip gradients over
the ranks in one all-reduce of 6N + 5 values.
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


GRAD_KEYS = ("x", "y", "z", "q", "R", "eps")
TIP_KEYS = ("kx", "ky", "kR", "Q", "Qzz")


def reduce_grads(grads: dict, device=None) -> dict:
    """Sum a gradient dict (per-atom arrays under GRAD_KEYS, scalars under TIP_KEYS; torch
    tensors or numpy arrays) over all ranks with one all-reduce of a packed float64 buffer.
    Returns a dict of the same keys (float64 torch tensors on the reduction device for the
    per-atom entries, Python floats for the scalars); without an initialised group it returns
    the input's values unchanged."""
    import torch.distributed as dist

    n = len(grads[GRAD_KEYS[0]])
    grouped = dist.is_available() and dist.is_initialized()
    if device is None:
        device = "cuda" if grouped and dist.get_backend() == "nccl" else "cpu"
    flat = torch.empty(6 * n + 5, dtype=torch.float64, device=device)
    for r, k in enumerate(GRAD_KEYS):
        v = grads[k]
        flat[r * n:(r + 1) * n] = v.to(device=device, dtype=torch.float64) if torch.is_tensor(v) else \
            torch.as_tensor(v, dtype=torch.float64, device=device)
    flat[6 * n:] = torch.tensor([float(grads.get(k, 0.0)) for k in TIP_KEYS], dtype=torch.float64, device=device)
    if grouped:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    out = {k: flat[r * n:(r + 1) * n] for r, k in enumerate(GRAD_KEYS)}
    out.update({k: float(flat[6 * n + i].item()) for i, k in enumerate(TIP_KEYS)})
    return out
