"""Host-side sharding of cells over ranks (one process per GPU).

Cells are independent problems (Sec. 2.1.3: one transform per cell), so a multi-GPU job splits the
cells over ranks and needs no collective on the data path.  The split balances the per-cell cost
16 Q + 8 P^2 bytes (samples read, coefficients written) by longest-processing-time-first assignment.
"""
from __future__ import annotations

import heapq

import numpy as np

__all__ = ["cell_cost", "partition_cells"]


def cell_cost(counts, modes: int) -> np.ndarray:
    """Bytes moved per cell: 16 B per sample in, 8 P^2 B of coefficients out."""
    return 16.0 * np.asarray(counts, dtype=np.float64) + 8.0 * modes * modes


def partition_cells(counts, modes: int, world_size: int) -> list[np.ndarray]:
    """Cell indices per rank (ascending), every cell on exactly one rank, costs balanced by LPT."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    cost = cell_cost(counts, modes)
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, r) for r in range(world_size)]
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for c in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(c))
        heapq.heappush(heap, (load + float(cost[c]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]
