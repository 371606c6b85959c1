"""Split a set of independent problems across ranks (one GPU each).

The problems of a batch share nothing, so a multi-GPU run needs no
communication on the data path: every rank advances its own subset in its own
persistent launch.  Subsets are balanced by cost (cells x steps) with the
longest-processing-time rule: problems in decreasing cost, each to the rank
with the least cost so far (ties to the lowest rank), which keeps the largest
rank within 4/3 of the optimum and, for thousands of small problems, within a
fraction of a percent of the mean.
"""
from __future__ import annotations

import heapq


def lpt_shards(costs, world):
    """Indices of `costs` per rank (lists sorted ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shards]


def spec_cost(spec):
    """Cost of one batched problem: cells times RK2 steps."""
    return spec.n ** spec.ndim * spec.steps


def weak_scaling_specs(world, per_rank=4096, seed=4):
    """The batched Riemann set for `world` ranks: `world` independent draws of
    `per_rank` problems (seeds seed .. seed + world - 1), so the work per GPU
    stays fixed as the rank count grows; world = 1 is the single-GPU set."""
    from . import problems as P
    specs = []
    for k in range(world):
        specs.extend(P.batched_riemann(count=per_rank, seed=seed + k))
    return specs


def rank_specs(specs, rank, world):
    """This rank's problems of `specs` (LPT by cells x steps)."""
    return [specs[i] for i in lpt_shards([spec_cost(s) for s in specs], world)[rank]]
