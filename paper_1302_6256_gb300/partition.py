"""Exact maximum clique over several ranks by a partition of the roots.

Section 4.5 of the paper spreads the roots of the neighbourhood search over
processors that share the incumbent.  Here each rank (one GPU per process)
holds the whole graph, computes the core numbers, the heuristic and the
pruning itself, and searches only the roots whose position in one shared
degeneracy order is congruent to its rank modulo the world size.  Every
clique has exactly one lowest-ranked member, so the parts cover every
clique once, and the largest clique over the ranks is omega.  The ranks
exchange twice: rank 0's peel order is broadcast before the search (the
peel order depends on timing, and every rank must orient the graph the same
way), and the (size, rank) of every rank's best clique is gathered after it;
the owner of the largest broadcasts its witness.

The local steps are passed in, so the same exchange runs over the CUDA
library (`library_steps`) or over any other implementation of the steps.
"""
from __future__ import annotations

import numpy as np


def partitioned_max_clique(peel_order, solve_part, rank: int, world: int, n: int, device="cpu", group=None):
    """omega of a graph whose roots are split over `world` ranks.

    peel_order() -> int32 array of n entries (called on rank 0 only): a
    degeneracy order of the graph.  solve_part(order, rank, world) ->
    (size, witness): the largest clique this rank's part of the roots finds
    (at least the heuristic's).  device: where the exchanged tensors live
    ("cpu" for gloo, a CUDA device for NCCL).  Returns (omega, witness,
    owner rank, list of every rank's size)."""
    import torch
    import torch.distributed as dist
    order = torch.empty(n, dtype=torch.int32, device=device)
    if rank == 0:
        order.copy_(torch.as_tensor(np.asarray(peel_order(), dtype=np.int32)))
    if world > 1:
        dist.broadcast(order, 0, group=group)
    size, wit = solve_part(order.cpu().numpy() if str(device) == "cpu" else order, rank, world)
    sizes = torch.zeros(world, dtype=torch.int64, device=device)
    sizes[rank] = int(size)
    if world > 1:
        dist.all_reduce(sizes, op=dist.ReduceOp.SUM, group=group)
    sizes = sizes.cpu().tolist()
    omega = max(sizes)
    owner = sizes.index(omega)  # the smallest rank among the largest
    w = torch.zeros(max(omega, 1), dtype=torch.int32, device=device)
    if rank == owner:
        w[:omega] = torch.as_tensor(np.asarray(wit, dtype=np.int32)[:omega])
    if world > 1:
        dist.broadcast(w, owner, group=group)
    return omega, w[:omega].cpu().numpy(), owner, sizes


def library_steps(g, **opts):
    """The local steps over the CUDA library for a loaded graph `g`: the
    peel order of its core numbers, and a solve restricted to one part."""
    from . import mc_core_numbers, mc_max_clique, mc_peel_order

    def peel_order():
        mc_core_numbers(g)
        return mc_peel_order(g)

    def solve_part(order, rank, world):
        om, wit, _ = mc_max_clique(g, order=order, part_rank=rank, part_count=world, **opts)
        return om, np.asarray(wit.cpu() if hasattr(wit, "cpu") else wit)

    return peel_order, solve_part
