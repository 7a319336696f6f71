"""Small shared helpers for the tests (dense matrices, random problems)."""
from __future__ import annotations

import numpy as np

from paper_1810_12742_gb300 import inputs as I


def dense(p, d, u):
    n = len(d)
    A = np.diag(np.asarray(d, np.float64))
    for i in range(1, n):
        A[i, p[i]] = u[i]
        A[p[i], i] = u[i]
    return A


def problem(p, rng, s_range=(0.01, 0.1)):
    """Coefficients on a given tree with the workload distributions."""
    n = len(p)
    a = rng.uniform(0.5, 2.0, n)
    a[0] = 0.0
    s = rng.uniform(*s_range, n)
    d = s + I.edge_sum(np.asarray(p), a)
    return dict(a=a, s=s, d=d, u=-a, b=rng.uniform(-1.0, 1.0, n))


def tree_zoo(rng, n):
    """A handful of differently shaped trees with n compartments."""
    out = {
        "chain": np.arange(-1, n - 1, dtype=np.int32),
        "recursive": I.random_recursive_tree(rng, n),
        "chainy": I.random_chainy_tree(rng, n, 0.15),
        "star": np.concatenate(([-1], np.zeros(max(n - 1, 0), np.int32))).astype(np.int32)[:n],
    }
    nb = max(1, n // 6)
    bp, _ = I.grow_branch_tree(rng, nb, 0.5, 0.2)
    lens = np.full(nb, n // nb)
    lens[: n - lens.sum()] += 1
    out["branchy"] = I.compartments_from_branches(bp, lens)
    return out


def relabel(p, rng):
    """A different valid Hines numbering of the same tree: random-order DFS
    preorder from the root.  Returns (new parent array, perm) with
    new index k holding old compartment perm[k]."""
    n = len(p)
    children = [[] for _ in range(n)]
    for i in range(1, n):
        children[p[i]].append(i)
    order, stack = [], [0]
    while stack:
        v = stack.pop()
        order.append(v)
        ch = list(children[v])
        rng.shuffle(ch)
        stack.extend(ch)
    perm = np.array(order)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    newp = np.full(n, -1, np.int32)
    for k in range(1, n):
        newp[k] = inv[p[perm[k]]]
    return newp, perm
