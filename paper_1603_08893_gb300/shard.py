"""Partition of independent cells over ranks (one process per GPU).

Cells of a batch are independent problems, so a multi-GPU run shards them
with no exchange in the data path: each rank solves its own cells and only
the timing and the totals are reduced.  The cost of a cell is taken as
n log2 n (n voxels; a CG iteration is a set of FFT passes), and cells are
assigned largest first to the least loaded rank (ties to the lower rank),
so every rank computes the same partition on its own.
"""
from __future__ import annotations

import math


def cell_cost(shape) -> float:
    n = 1
    for s in shape:
        n *= int(s)
    return n * math.log2(max(n, 2))


def partition_cells(shapes, world: int):
    """List of `world` lists of cell indices (each ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(shapes)), key=lambda i: (-cell_cost(shapes[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += cell_cost(shapes[i])
    return [sorted(p) for p in parts]
