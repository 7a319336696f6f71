"""Re-rooting at the centre (Section 6, balancing the dependency tree): the
C++ planner's new roots and renumbering must agree bit for bit with an
independent Python statement; the new root must minimise the depth (brute
force on small trees); and the re-rooted system, solved by the oracle and
mapped back, must give the original solution (host-only plans, no GPU)."""
import numpy as np
import pytest

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I
from tests.helpers import dense, problem, tree_zoo


def py_eccentricity(p):
    """Largest distance (edges) from each compartment to any other, by the two
    passes of tree dynamic programming: heights below each compartment, then
    the longest path that leaves it through its parent."""
    n = len(p)
    down = np.zeros(n, np.int64)
    for i in range(n - 1, 0, -1):
        down[p[i]] = max(down[p[i]], down[i] + 1)
    best = np.full((n, 2), -1, np.int64)  # two largest down[child] + 1 per compartment
    for i in range(1, n):
        h = down[i] + 1
        v = p[i]
        if h > best[v, 0]:
            best[v, 1], best[v, 0] = best[v, 0], h
        elif h > best[v, 1]:
            best[v, 1] = h
    up = np.zeros(n, np.int64)
    for i in range(1, n):
        v = p[i]
        other = best[v, 1] if down[i] + 1 == best[v, 0] else best[v, 0]
        up[i] = 1 + max(up[v], other if other > 0 else 0)
    return np.maximum(down, up)


def brute_eccentricity(p):
    n = len(p)
    adj = [[] for _ in range(n)]
    for i in range(1, n):
        adj[i].append(p[i])
        adj[p[i]].append(i)
    ecc = np.empty(n, np.int64)
    for s in range(n):
        dist = {s: 0}
        frontier = [s]
        while frontier:
            nxt = []
            for x in frontier:
                for y in adj[x]:
                    if y not in dist:
                        dist[y] = dist[x] + 1
                        nxt.append(y)
            frontier = nxt
        ecc[s] = max(dist.values())
    return ecc


def py_reroot(p):
    """(new parent, perm, edge, centre) of one cell: root at the smallest-index
    compartment of least eccentricity; branches numbered breadth first from the
    root branch, each proximal to distal, children in ascending old index."""
    n = len(p)
    if n == 0:
        return (np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.int64), 0)
    c = int(np.argmin(py_eccentricity(p)))
    adj = [[] for _ in range(n)]
    for i in range(1, n):
        adj[i].append(p[i])
        adj[p[i]].append(i)
    newp_old = np.full(n, -1, np.int64)
    seen = np.zeros(n, bool)
    seen[c] = True
    order = [c]
    for x in order:
        for y in adj[x]:
            if not seen[y]:
                seen[y] = True
                newp_old[y] = x
                order.append(y)
    kids = [sorted(y for y in adj[x] if y != newp_old[x]) for x in range(n)]
    perm, starts = [], [c]
    for s in starts:
        x = s
        while True:
            perm.append(x)
            if len(kids[x]) == 1:
                x = kids[x][0]
                continue
            starts.extend(kids[x])
            break
    perm = np.array(perm, np.int64)
    new_of = np.empty(n, np.int64)
    new_of[perm] = np.arange(n)
    newp = np.array([-1 if newp_old[x] < 0 else new_of[newp_old[x]] for x in perm], np.int32)
    edge = np.array([-1 if newp_old[x] < 0 else (x if p[x] == newp_old[x] else newp_old[x]) for x in perm], np.int64)
    return newp, perm, edge, c


def _batch(trees):
    ncomp = np.array([t.size for t in trees], np.int32)
    return ncomp, (np.concatenate(trees) if trees else np.zeros(0, np.int32)).astype(np.int32)


def _compare(ncomp, parent):
    plan = H.Plan(ncomp, parent, host_only=True, reroot=True)
    got = plan.export_reroot()
    off = np.concatenate(([0], np.cumsum(ncomp))).astype(np.int64)
    for c in range(ncomp.size):
        sl = slice(off[c], off[c + 1])
        newp, perm, edge, centre = py_reroot(parent[sl])
        assert got["centre"][c] == centre
        assert np.array_equal(got["parent"][sl], newp)
        assert np.array_equal(got["perm"][sl], perm + off[c])
        assert np.array_equal(got["edge"][sl], np.where(edge >= 0, edge + off[c], -1))
    # the plan describes the re-rooted morphology
    ref = H.Plan(ncomp, got["parent"], host_only=True)
    assert np.array_equal(plan.export()["first"], ref.export()["first"])
    # its solver layout maps onto the caller's numbering
    slots = plan.export_packed()
    ref_slots = ref.export_packed()
    assert np.array_equal(slots, np.where(ref_slots >= 0, got["perm"][np.maximum(ref_slots, 0)], -1))
    return got


def test_eccentricity_statement_matches_brute_force():
    rng = np.random.default_rng(3)
    for n in (1, 2, 3, 7, 40, 150):
        for p in tree_zoo(rng, n).values():
            assert np.array_equal(py_eccentricity(p), brute_eccentricity(p))


def test_zoo_matches_restatement():
    rng = np.random.default_rng(17)
    trees = []
    for n in (1, 2, 3, 4, 9, 33, 250, 3000):
        trees += list(tree_zoo(rng, n).values())
    _compare(*_batch(trees))


@pytest.mark.parametrize("name", ["fp64_small", "fp64_uniform", "uneven_steps"])
def test_workload_samples_match_restatement(name):
    w = I.WORKLOADS[name]
    cells = np.arange(min(w.n_cells, 12))
    if name == "uneven_steps":
        cls = I.cell_classes(w)
        cells = np.concatenate([np.nonzero(cls == 0)[0][:4], np.nonzero(cls == 1)[0][:2]])
    ncomp, parent = I.population_trees(w, cells)
    _compare(ncomp, parent)


def test_new_root_minimises_depth_and_order_is_hines():
    rng = np.random.default_rng(8)
    trees = []
    for n in (2, 5, 30, 120):
        trees += list(tree_zoo(rng, n).values())
    ncomp, parent = _batch(trees)
    got = H.Plan(ncomp, parent, host_only=True, reroot=True).export_reroot()
    off = np.concatenate(([0], np.cumsum(ncomp)))
    for c in range(ncomp.size):
        sl = slice(off[c], off[c + 1])
        ecc = brute_eccentricity(parent[sl])
        newp = got["parent"][sl]
        assert newp[0] == -1 and all(0 <= newp[i] < i for i in range(1, newp.size))
        depth = np.zeros(newp.size, np.int64)
        for i in range(1, newp.size):
            depth[i] = depth[newp[i]] + 1
        assert depth.max() == ecc.min() <= ecc[0]  # the radius, never deeper than before
        assert got["centre"][c] == np.flatnonzero(ecc == ecc.min()).min()
        # each undirected edge keeps its coupling: {perm[i], perm[p'(i)]} is an old edge stored at edge[i]
        perm = got["perm"][sl] - off[c]
        edge = got["edge"][sl] - off[c]
        for i in range(1, newp.size):
            a, b = perm[i], perm[newp[i]]
            assert (parent[sl][a] == b and edge[i] == a) or (parent[sl][b] == a and edge[i] == b)


def test_rerooted_system_has_the_same_solution():
    """Oracle pin: the re-rooted Hines system (d, b through perm, couplings
    through edge) solved by the oracle and mapped back equals the original
    solution, and both equal dense LU."""
    rng = np.random.default_rng(23)
    trees = [t for n in (1, 2, 6, 40, 180) for t in tree_zoo(rng, n).values()]
    ncomp, parent = _batch(trees)
    got = H.Plan(ncomp, parent, host_only=True, reroot=True).export_reroot()
    off = np.concatenate(([0], np.cumsum(ncomp)))
    for c in range(ncomp.size):
        sl = slice(off[c], off[c + 1])
        p = parent[sl]
        pr = problem(p, rng)
        x = oracle.hines(p, pr["d"], pr["u"], pr["b"])
        perm = got["perm"][sl] - off[c]
        edge = got["edge"][sl] - off[c]
        ur = np.where(edge >= 0, pr["u"][np.maximum(edge, 0)], 0.0)
        y = oracle.hines(got["parent"][sl], pr["d"][perm], ur, pr["b"][perm])
        back = np.empty_like(y)
        back[perm] = y
        ref = np.linalg.solve(dense(p, pr["d"], np.where(np.arange(p.size) > 0, pr["u"], 0.0)), pr["b"])
        scale = np.abs(ref).max()
        assert np.abs(back - x).max() <= 1e-13 * scale
        assert np.abs(back - ref).max() <= 1e-12 * scale


def test_export_reroot_needs_a_rerooted_plan():
    ncomp, parent = _batch([np.array([-1, 0, 1], np.int32)])
    with pytest.raises(H.HinesError):
        H.Plan(ncomp, parent, host_only=True).export_reroot()
    with pytest.raises(H.HinesError):  # validation still applies
        H.Plan(ncomp, np.array([-1, 2, 0], np.int32), host_only=True, reroot=True)


def test_empty_cells_and_batches():
    plan = H.Plan(np.zeros(0, np.int32), np.zeros(0, np.int32), host_only=True, reroot=True)
    assert plan.n_unknowns == 0 and plan.export_reroot()["perm"].size == 0
    ncomp = np.array([0, 1, 0, 3], np.int32)
    parent = np.array([-1, -1, 0, 1], np.int32)
    got = _compare(ncomp, parent)
    assert got["perm"].tolist() == [0, 2, 1, 3]  # the chain 1-2-3 re-rooted at its middle
    assert got["edge"].tolist() == [-1, -1, 2, 3]
    assert got["parent"].tolist() == [-1, -1, 0, 0]
