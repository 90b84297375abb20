"""Partition of independent objects over ranks (one process per GPU).

Every object is trained on its own (the paper runs one mapping thread per
object, §IV-A), so a multi-GPU step splits the objects between the ranks and
exchanges nothing on the data path: each rank trains its share with one
batched training step, and only the timing is reduced afterwards.

The split is longest-processing-time first (Graham, "Bounds on
multiprocessing timing anomalies", 1969): objects in order of decreasing
cost, each given to the rank with the smallest load so far.  Its makespan is
at most 4/3 - 1/(3 world) of the optimum.  Ties are broken by object index and
rank number, so every rank computes the same partition from the same list.
"""

from __future__ import annotations

from typing import List, Sequence


def object_cost(L: int, F: int, width: int, hidden: int, n_params: int, n_samples: int,
                feature_bytes: int = 4) -> float:
    """Cost of one training step of one object, in byte-equivalents: per sample
    the hash gather and scatter (8 corners x L levels x F features, read in
    `feature_bytes` and added back in FP32) plus two operations per MLP
    multiply-add, and 28 bytes of the Adam pass per parameter."""
    if min(L, F, width, hidden) < 1 or n_params < 0 or n_samples < 0:
        raise ValueError("object_cost: sizes must be positive")
    macs = width * L * F + (hidden - 1) * width * width + 4 * width
    per_sample = 8 * L * F * (feature_bytes + 4) + 2 * macs
    return float(n_samples) * per_sample + 28.0 * n_params


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Object indices of each rank (each list in increasing index order)."""
    if world < 1:
        raise ValueError("lpt_partition: world must be >= 1")
    if any(c < 0 for c in costs):
        raise ValueError("lpt_partition: costs must be non-negative")
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def rank_objects(costs: Sequence[float], world: int, rank: int) -> List[int]:
    """The objects this rank trains."""
    if not 0 <= rank < world:
        raise ValueError("rank_objects: rank out of range")
    return lpt_partition(costs, world)[rank]


def makespan(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> float:
    return max((sum(costs[i] for i in p) for p in parts), default=0.0)
