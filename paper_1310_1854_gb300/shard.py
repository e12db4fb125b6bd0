"""Ray sharding over several processes (one per GPU).

Rays are independent (Sect. 2.2 traces each path on its own), so the forward
pass splits the rays across ranks with the grid replicated and needs no
exchange; results stay on the rank that traced them. The adjoint is the one
place with a real exchange: every rank adds its rays' contributions to the
same per-cell gradient, so the partial gradients are summed across ranks.
These helpers work with any torch.distributed backend (NCCL on GPUs, gloo
for the CPU tests).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) block of n items for `rank` of `world`; the
    first n % world ranks get one extra item."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def allreduce_sum_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum across ranks (no-op without an initialised group)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def max_over_ranks(x: float, device=None, group=None) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(x: float, device=None, group=None) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def sharded_density_grad(grid, origin, direction, dL_dtau, group=None):
    """dL/drho over all ranks' rays: each rank runs the adjoint traversal on
    its own rays, then the per-cell partial gradients are summed."""
    g = grid.trace_grad(origin, direction, dL_dtau)
    return allreduce_sum_(g, group)
