"""Seeded synthetic inputs for the batched Hines solver.

This module only draws random tree shapes and random coefficients; it contains
no solver arithmetic and imports neither the CUDA binding nor the oracle, so
the tests, the bench and the oracle checks can all share it.

Workload recipe (the paper's own benchmark is the ring-network example of the
Arbor simulator, Section 7, which is not available here; these synthetic
populations stand in for it and mimic its structure: random dendritic trees
grown level by level with a split probability and random branch lengths):

* Trees are grown per branch.  A pass visits the current leaf branches in
  creation order; each leaf (below the depth cap) splits with probability
  ``p_split`` into 3 children with probability ``p_ternary``, else 2.  Two
  uniforms are drawn per visited leaf (split, arity), always, in that order.
  Passes repeat until the branch count is reached exactly: a split that would
  overshoot is trimmed to the branches still missing, and if exactly one is
  missing it is attached as an extra child of the most recent split.
* Branches are renumbered breadth first (by level, then by the new index of
  the parent, then by creation order) and each gets a compartment count drawn
  uniformly (inclusive bounds).  Compartments are numbered branch by branch,
  proximal to distal, so the parent of a branch's first compartment is the
  last compartment of its parent branch and p[i] < i holds (Hines order,
  Section 2 of the paper).
* Coefficients: one axial conductance a_i ~ U[0.5, 2] per edge (i, p[i]);
  the leak/capacitance term s_i ~ U[0.01, 0.1] (or U[0.1 m, m] for a margin m);
  off-diagonal u_i = -a_i (u_0 = 0); diagonal d_i = s_i + sum of the a over the
  edges at i (the finite-volume system of Section 1, eq. for V^{k+1});
  right-hand side b_i ~ U[-1, 1].
* Every cell draws from its own numpy PCG64 stream seeded with
  (12742 + config, cell, purpose), so any subset of cells can be regenerated.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 12742


# ----------------------------------------------------------------------------
# tree shapes
# ----------------------------------------------------------------------------
def grow_branch_tree(rng: np.random.Generator, n_branches: int, p_split: float = 0.5,
                     p_ternary: float = 0.0, depth_cap: int | None = None):
    """Random branch tree with exactly ``n_branches`` branches.

    Returns (branch_parent, branch_level), both int32 and breadth-first
    numbered (branch 0 is the root branch, parent index < child index).
    """
    if n_branches < 1:
        raise ValueError("n_branches must be >= 1")
    parent = np.full(n_branches, -1, np.int64)
    level = np.zeros(n_branches, np.int64)
    frontier = np.zeros(1, np.int64)
    count = 1
    last_split = -1
    while count < n_branches:
        F = frontier
        u_split = rng.random(F.size)
        u_arity = rng.random(F.size)
        lv = level[F]
        can = np.ones(F.size, bool) if depth_cap is None else lv < depth_cap
        if not can.any():
            raise ValueError("depth cap reached before the branch count")
        split = can & (u_split < p_split)
        arity = np.where(split, np.where(u_arity < p_ternary, 3, 2), 0)
        need = n_branches - count
        csum = np.cumsum(arity)
        extra_parent = -1
        if csum.size and csum[-1] >= need:
            cut = int(np.searchsorted(csum, need))          # first index with csum >= need
            before = int(csum[cut] - arity[cut])
            rem = need - before
            arity[cut + 1:] = 0
            if rem >= 2:
                arity[cut] = rem
            else:                                            # exactly one branch missing
                arity[cut] = 0
                prev = np.nonzero(arity[:cut] > 0)[0]
                extra_parent = int(F[prev[-1]]) if prev.size else last_split
                if extra_parent < 0:                         # no split yet: root gets one child
                    extra_parent = 0
        n_new = int(arity.sum())
        if n_new:
            new_ids = count + np.arange(n_new)
            parent[new_ids] = np.repeat(F, arity)
            level[new_ids] = np.repeat(lv + 1, arity)
            last_split = int(F[np.nonzero(arity)[0][-1]])
            cnt = np.where(arity > 0, arity, 1)
            nf = np.repeat(F, cnt)
            nf[np.repeat(arity > 0, cnt)] = new_ids
            frontier = nf
            count += n_new
        if extra_parent >= 0:
            parent[count] = extra_parent
            level[count] = level[extra_parent] + 1
            frontier = np.append(frontier, count)
            last_split = extra_parent
            count += 1
    # breadth-first renumbering: by level, then new index of parent, then creation order
    new_index = np.empty(n_branches, np.int64)
    order_all = []
    new_index[0] = 0
    order_all.append(np.zeros(1, np.int64))
    nxt = 1
    max_level = int(level.max())
    for lvl in range(1, max_level + 1):
        ids = np.nonzero(level == lvl)[0]
        o = np.lexsort((ids, new_index[parent[ids]]))
        ids = ids[o]
        new_index[ids] = nxt + np.arange(ids.size)
        nxt += ids.size
        order_all.append(ids)
    order = np.concatenate(order_all)                        # old ids in new order
    bparent = np.where(parent[order] >= 0, new_index[np.maximum(parent[order], 0)], -1)
    return bparent.astype(np.int32), level[order].astype(np.int32)


def compartments_from_branches(branch_parent: np.ndarray, branch_len: np.ndarray) -> np.ndarray:
    """Compartment parent array (Hines order) from a BFS branch tree and branch lengths."""
    branch_len = np.asarray(branch_len, np.int64)
    if (branch_len < 1).any():
        raise ValueError("every branch needs at least one compartment")
    first = np.concatenate(([0], np.cumsum(branch_len)[:-1]))
    last = first + branch_len - 1
    n = int(branch_len.sum())
    p = np.arange(n, dtype=np.int64) - 1
    bp = np.asarray(branch_parent, np.int64)
    p[first] = np.where(bp >= 0, last[np.maximum(bp, 0)], -1)
    return p.astype(np.int32)


def random_recursive_tree(rng: np.random.Generator, n: int) -> np.ndarray:
    """Parent array with p[i] ~ U{0..i-1}: many branch points, short branches."""
    p = np.empty(n, np.int32)
    p[0] = -1
    if n > 1:
        p[1:] = np.floor(rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
    return p


def random_chainy_tree(rng: np.random.Generator, n: int, p_branch: float = 0.1) -> np.ndarray:
    """Parent array that mostly continues the chain (p[i] = i-1) and sometimes
    attaches anywhere earlier (p[i] ~ U{0..i-1}), including mid-branch."""
    p = random_recursive_tree(rng, n)
    if n > 1:
        cont = rng.random(n - 1) >= p_branch
        idx = np.arange(1, n)
        p[1:] = np.where(cont, idx - 1, p[1:])
    return p


# ----------------------------------------------------------------------------
# workload configurations
# ----------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class CellClass:
    branches: tuple[int, int]        # inclusive U[lo, hi] branch count
    lengths: tuple[int, int]         # inclusive U[lo, hi] compartments per branch
    p_split: float = 0.5
    p_ternary: float = 0.1
    depth_cap: int | None = None


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    cfg: int                          # index used in the seed
    tree_cfg: int                     # seed index of the tree shapes (shared populations)
    n_cells: int
    classes: tuple[CellClass, ...]
    class_frac: tuple[float, ...]     # fraction of cells in each class (exact counts, seeded placement)
    s_range: tuple[float, float] = (0.01, 0.1)
    steps: int = 0
    dt: float = 0.025
    E: float = -65.0
    checkpoint_every: int = 0


_C0 = CellClass(branches=(31, 31), lengths=(8, 8), p_split=0.5, p_ternary=0.0)
_C1 = CellClass(branches=(100, 300), lengths=(4, 32), p_split=0.5, p_ternary=0.1)
_C2S = CellClass(branches=(50, 200), lengths=(4, 16), p_split=0.5, p_ternary=0.1, depth_cap=40)
_C2L = CellClass(branches=(1000, 4000), lengths=(8, 64), p_split=0.5, p_ternary=0.1, depth_cap=40)
_C4 = CellClass(branches=(100, 500), lengths=(16, 16), p_split=0.5, p_ternary=0.1)

WORKLOADS = {
    "fp64_small": Workload("fp64_small: 64 binary cells x 31 branches x 8 compartments", 0, 0, 64, (_C0,), (1.0,)),
    "fp64_uniform": Workload("fp64_uniform: 16384 cells, U[100,300] branches x U[4,32] compartments", 1, 1,
                             16384, (_C1,), (1.0,)),
    "uneven_steps": Workload("uneven_steps: 8192 cells (70% small, 30% large), passive cable, 1000 steps", 2, 2,
                             8192, (_C2S, _C2L), (0.7, 0.3), steps=1000),
    "uneven_mixed": Workload("uneven_mixed: 8192 cells (70% small, 30% large), FP32 d, u, b in, FP64 x out", 3, 2,
                             8192, (_C2S, _C2L), (0.7, 0.3)),
    "adjoint": Workload("adjoint: 256 cells x U[100,500] branches x 16 compartments, 200 steps", 4, 4,
                        256, (_C4,), (1.0,), steps=200, checkpoint_every=20),
}
MARGINS = (1e-1, 1e-3, 1e-5)


def _rng(cfg: int, cell: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + cfg, cell, purpose])


def cell_classes(w: Workload) -> np.ndarray:
    """Class index of every cell: exact counts per class, seeded placement."""
    counts = [int(round(f * w.n_cells)) for f in w.class_frac]
    counts[0] = w.n_cells - sum(counts[1:])
    cls = np.concatenate([np.full(c, i, np.int32) for i, c in enumerate(counts)])
    return np.random.default_rng([SEED_BASE + w.tree_cfg, 1 << 30]).permutation(cls)


def cell_tree(w: Workload, cell: int, cls: int | None = None) -> np.ndarray:
    if cls is None:
        cls = int(cell_classes(w)[cell])
    c = w.classes[cls]
    rng = _rng(w.tree_cfg, cell, 0)
    nb = int(rng.integers(c.branches[0], c.branches[1] + 1))
    bp, _ = grow_branch_tree(rng, nb, c.p_split, c.p_ternary, c.depth_cap)
    lens = rng.integers(c.lengths[0], c.lengths[1] + 1, size=nb)
    return compartments_from_branches(bp, lens)


def population_trees(w: Workload, cells=None):
    """(ncomp int32[n], parent int32[sum ncomp]) for the chosen cells (default all)."""
    cells = np.arange(w.n_cells) if cells is None else np.asarray(cells)
    cls = cell_classes(w)
    trees = [cell_tree(w, int(c), int(cls[c])) for c in cells]
    ncomp = np.array([t.size for t in trees], np.int32)
    parent = np.concatenate(trees) if trees else np.zeros(0, np.int32)
    return ncomp, parent


def edge_sum(parent: np.ndarray, a: np.ndarray) -> np.ndarray:
    """sum over the edges at each compartment of a per-edge value a[i] (edge i -> p[i])."""
    n = parent.size
    out = np.zeros(n, np.float64)
    if n > 1:
        out[1:] += a[1:]
        out += np.bincount(parent[1:], weights=a[1:], minlength=n)
    return out


def cell_coefficients(w: Workload, cell: int, parent: np.ndarray, margin: float | None = None,
                      purpose: int = 1) -> dict:
    """Coefficients of one cell (float64).  Keys: a, s, u, d, b, and for
    time-stepping workloads g, V0 and the scalar target."""
    n = parent.size
    rng = _rng(w.cfg, cell, purpose)
    a = rng.uniform(0.5, 2.0, size=n)
    a[0] = 0.0
    lo, hi = (w.s_range if margin is None else (0.1 * margin, margin))
    s = rng.uniform(lo, hi, size=n)
    b = rng.uniform(-1.0, 1.0, size=n)
    out = dict(a=a, s=s, u=-a, d=s + edge_sum(parent, a), b=b)
    if w.steps:
        out["g"] = rng.uniform(0.1, 1.0, size=n)
        out["V0"] = rng.uniform(-80.0, -50.0, size=n)
        out["target"] = float(rng.uniform(-70.0, -50.0))
    return out


def population(w: Workload | str, cells=None, margin: float | None = None, keys=("d", "u", "b")) -> dict:
    """Whole (or partial) population in natural layout: cells concatenated in
    the order given.  Returns ncomp, parent, offsets (int64[n+1]) and the
    requested coefficient arrays (float64), plus 'target' (per cell) when the
    workload steps in time and 'target' is requested."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    cells = np.arange(w.n_cells) if cells is None else np.asarray(cells)
    ncomp, parent = population_trees(w, cells)
    off = np.zeros(ncomp.size + 1, np.int64)
    np.cumsum(ncomp, out=off[1:])
    out = dict(ncomp=ncomp, parent=parent, offsets=off, cells=cells)
    arrays = {k: np.empty(int(off[-1]), np.float64) for k in keys if k != "target"}
    targets = np.empty(ncomp.size, np.float64)
    for j, c in enumerate(cells):
        lo, hi = int(off[j]), int(off[j + 1])
        co = cell_coefficients(w, int(c), parent[lo:hi], margin)
        for k in arrays:
            arrays[k][lo:hi] = co[k]
        if "target" in keys:
            targets[j] = co["target"]
    out.update(arrays)
    if "target" in keys:
        out["target"] = targets
    return out
