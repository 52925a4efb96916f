"""Multi-GPU sharding of the fitness path (host logic).

The fitness of a population shards two ways without changing any result
beyond rounding:
  * by population: trees are independent, each rank evaluates a contiguous
    range of trees (no exchange on the data path; `population_range`);
  * by points: each rank evaluates every tree on a contiguous range of
    points and the per-tree sums of squared residuals are added across
    ranks (one all-reduce of pop * n_outputs doubles; `combine_point_shards`).
The benchmark uses population replicas (weak scaling).  The point-sharded
combination is what a rank-parallel caller runs: each rank calls
tgp_fitness_mse_cfg with the TGP_FLAG_SSE flag, which returns the FP64 sum of
squared residuals over its points (no division), then
    SSE = all_reduce(sum, sse_r);  MSE = SSE / D_total.

A generation (Algorithm 1) shards its fitness by population and replicates
the rest: each rank evaluates its range of trees, one all-gather of P
doubles gives every rank the whole fitness vector (`gather_fitness`), and
every rank then runs selection, crossover and mutation on the replicated
population with the same random words, so the populations stay identical
without moving any tree between ranks (the operators cost well under 1% of
the fitness).
"""
from __future__ import annotations


def population_range(pop: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) of trees owned by `rank` (sizes differ by <= 1)."""
    base, rem = divmod(pop, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)


def point_range(n_points: int, rank: int, world: int) -> tuple[int, int]:
    return population_range(n_points, rank, world)


def combine_point_shards(sse_local, n_total: int, group=None):
    """MSE over all points from each rank's sum of squared residuals over its
    own points (the TGP_FLAG_SSE output of tgp_fitness_mse_cfg; a rank with
    no points passes zeros).

    `sse_local` is a float64 tensor [pop, n_outputs] (NaN rows of invalid trees
    stay NaN).  Uses one torch.distributed all_reduce (sum)."""
    import torch
    import torch.distributed as dist
    sse = sse_local.to(torch.float64).clone()
    dist.all_reduce(sse, op=dist.ReduceOp.SUM, group=group)
    return sse / float(n_total)


def gather_fitness(fit_local, pop: int, group=None):
    """The whole population's fitness on every rank from each rank's slice
    (its `population_range`): one all-gather, padded to the largest slice."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [b - a for a, b in (population_range(pop, r, world) for r in range(world))]
    width = max(sizes) if sizes else 0
    pad = torch.full((width,) + tuple(fit_local.shape[1:]), float("nan"), dtype=fit_local.dtype,
                     device=fit_local.device)
    pad[:fit_local.shape[0]] = fit_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:n] for p, n in zip(parts, sizes)])
