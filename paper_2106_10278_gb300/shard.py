"""Spreading the estimator over processes (one per GPU).

The estimator of eq. NPCF-estimator-discrete is a sum over primaries, so work
splits two ways:

* one catalogue: every rank holds all particles (they are all secondaries)
  and takes a contiguous range of primaries; the FP64 partial coefficients are
  summed with a single all-reduce -- the only exchange step;
* a batch of independent catalogues: whole catalogues go to ranks by
  longest-processing-time-first on their estimated pair counts; nothing is
  exchanged until the per-catalogue results are gathered.

These helpers only decide who computes what and move the results; the
coefficients themselves come from the `compute` callables (on a GPU,
Plan.compute / Plan.compute_batched).
"""
from __future__ import annotations

import math

import numpy as np


def primary_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous primary ranges [pb, pe) covering 0..n, sizes differing by at most one."""
    if world < 1 or n < 0:
        raise ValueError("world >= 1 and n >= 0 required")
    base, extra = divmod(n, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def sharded_compute(compute, n: int, group=None):
    """This rank's share of one catalogue, summed over all ranks.

    compute(pb, pe) -> float64 tensor (re, im interleaved) of the coefficients
    of primaries [pb, pe).  Returns the full coefficients on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    pb, pe = primary_ranges(n, world)[rank]
    part = compute(pb, pe)
    dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def estimated_pairs(sizes, boxes, edges, D: int) -> np.ndarray:
    """Expected ordered pairs of each catalogue if it were uniform: n^2 v_shell / V."""
    sizes = np.asarray(sizes, dtype=np.float64)
    boxes = np.asarray(boxes, dtype=np.float64).reshape(len(sizes), -1)
    area = 2.0 * math.pi ** (D / 2) / math.gamma(D / 2)
    shell = area / D * (float(edges[-1]) ** D - float(edges[0]) ** D)
    return sizes * sizes * shell / np.prod(boxes, axis=1)


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Longest processing time first: catalogues by decreasing cost (ties by index), each to the
    least-loaded rank (ties to the lowest rank).  Deterministic on every rank."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    for lst in out:
        lst.sort()
    return out


def sharded_batch(compute_one, costs, group=None) -> list:
    """Catalogues spread over ranks by lpt_assign; compute_one(i) -> CPU tensor of catalogue i's
    coefficients.  Returns every catalogue's result, in catalogue order, on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = lpt_assign(costs, world)[rank]
    local = {i: compute_one(i) for i in mine}
    every = [None] * world
    dist.all_gather_object(every, local, group=group)
    merged = {}
    for d in every:
        merged.update(d)
    return [merged[i] for i in range(len(costs))]
