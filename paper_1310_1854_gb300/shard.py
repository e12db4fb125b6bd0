"""Ray sharding over several processes (one per GPU).

Rays are independent (Sect. 2.2 traces each path on its own), so the forward
pass splits the rays across ranks with the grid replicated and needs no
exchange; results stay on the rank that traced them. A batch of many grids
is split by whole grids instead, each rank taking a set of grids whose
estimated crossings add up to about the same work. The adjoint is the one
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


def estimated_crossings(n_rays: int, n_sites: int) -> float:
    """Relative work of tracing n_rays through a grid of n_sites sites in a
    box of fixed size: the faces a line crosses per unit length grow as the
    cube root of the site density, so crossings ~ n_rays n_sites^(1/3)."""
    return float(n_rays) * float(max(n_sites, 1)) ** (1.0 / 3.0)


def assign_sets(weights, world: int) -> list[int]:
    """Rank of each set (grid and its rays) of a batch, for `world` ranks:
    the sets are taken heaviest first and each goes to the rank with the
    least work so far (ties to the lower rank). Deterministic, so every rank
    computes the same assignment without an exchange; the most loaded rank
    carries at most 4/3 of the optimum (the bound of this greedy rule)."""
    if world < 1:
        raise ValueError("world size must be at least 1")
    w = [float(x) for x in weights]
    if any(x < 0 for x in w):
        raise ValueError("weights must be non-negative")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    load = [0.0] * world
    out = [0] * len(w)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[i] = r
        load[r] += w[i]
    return out
