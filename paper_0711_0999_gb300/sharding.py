"""Host-side sharding across ranks (one process per GPU).

The quadrature points of a lattice step are independent (Sec. II: the sum of
Eq. g_loc over the (eps, ebar) grid), so a step shards by contiguous,
count-balanced blocks of points: each rank runs the lattice step on its
block and the partial G_loc and j(t) are summed.  The sum is made
deterministic by gathering every rank's partial and adding them in rank
order (no reduction tree whose order depends on the collective library).
Independent runs (several (U, E, dt)) shard by run with no collective at all.

This module only partitions, gathers and reduces; every arithmetic step of a
lattice step runs in the CUDA library.
"""

from __future__ import annotations

import torch
import torch.distributed as dist


def block_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of the rank's contiguous block when n items are split into
    `world` blocks whose sizes differ by at most one (the first n % world
    blocks are one larger)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad partition n={n} world={world} rank={rank}")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def ordered_sum(partial: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of every rank's `partial` (same shape and dtype on every rank),
    added in rank order 0, 1, ... on every rank; complex tensors travel as
    their real view."""
    world = dist.get_world_size(group)
    if world == 1:
        return partial.clone()
    x = torch.view_as_real(partial).contiguous() if partial.is_complex() else partial.contiguous()
    parts = [torch.empty_like(x) for _ in range(world)]
    dist.all_gather(parts, x, group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return torch.view_as_complex(out) if partial.is_complex() else out


def max_over_ranks(value: float, device, group=None) -> float:
    """The largest `value` over the ranks (the job's time is its slowest rank's)."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def lattice_gloc_sharded(grid, model, sigma, eps, ebar, wq, precision="mixed_bf16", group=None):
    """One lattice step with the points split over the ranks of `group`:
    (G_loc, j, j_imag) summed over all points, identical on every rank."""
    from . import api

    world, rank = dist.get_world_size(group), dist.get_rank(group)
    lo, hi = block_range(len(wq), world, rank)
    if hi > lo:
        gl, j, ji = api.lattice_gloc(grid, model, sigma, eps[lo:hi], ebar[lo:hi], wq[lo:hi], precision=precision)
    else:
        dev = sigma.device
        gl = torch.zeros((grid.n_c, grid.n_c), dtype=torch.complex128, device=dev)
        j = torch.zeros(grid.n_t, dtype=torch.float64, device=dev)
        ji = torch.zeros_like(j)
    return ordered_sum(gl, group), ordered_sum(j, group), ordered_sum(ji, group)
