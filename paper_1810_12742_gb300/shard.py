"""Cells across ranks: one process per GPU, each solving its own cells.

Cells are independent systems, so a batch splits across GPUs with no exchange
on the data path: every rank builds a plan for its cells and solves them.
The split balances the ranks' work by the longest-processing-time rule --
cells by compartments descending (ties by index), each to the rank with the
least work so far (ties by rank) -- which the solve time follows (a solve is
bound by the compartments it streams).  Every rank computes the same split
from the same compartment counts, so no rank has to send it.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(ncomp, n_parts: int) -> list[np.ndarray]:
    """Cell indices of each part (ascending within a part)."""
    if n_parts < 1:
        raise ValueError(f"n_parts: expected >= 1, got {n_parts}")
    nc = np.asarray(ncomp, np.int64)
    order = np.lexsort((np.arange(nc.size), -nc))  # compartments descending, then index
    heap = [(0, r) for r in range(n_parts)]
    parts = [[] for _ in range(n_parts)]
    for c in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(c))
        heapq.heappush(heap, (load + int(nc[c]), r))
    return [np.array(sorted(p), np.int64) for p in parts]


def shard_loads(ncomp, parts) -> np.ndarray:
    """Compartments per part."""
    nc = np.asarray(ncomp, np.int64)
    return np.array([int(nc[p].sum()) for p in parts], np.int64)
