"""Host planner: an independent Python statement of the decomposition,
splitting and ordering rules must agree bit for bit with the C++ planner
(host-only plans, no GPU needed)."""
import heapq

import numpy as np
import pytest

from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I
from tests.helpers import tree_zoo


def py_branches(p):
    """Branches of one cell: maximal runs i, i+1, ... where each next
    compartment's parent is its predecessor and that predecessor has one child."""
    n = len(p)
    nchild = np.bincount(np.asarray(p[1:], np.int64), minlength=n) if n > 1 else np.zeros(n, np.int64)
    br = []  # [first, len, parent_branch, level]
    owner = np.empty(n, np.int64)
    for i in range(n):
        if i == 0 or p[i] != i - 1 or nchild[p[i]] >= 2:
            pb = -1 if i == 0 else int(owner[p[i]])
            br.append([i, 1, pb, 0 if pb < 0 else br[pb][3] + 1])
        else:
            br[-1][1] += 1
        owner[i] = len(br) - 1
    return br


def py_split(cells, local=False):
    """Section 6 splitting: per level, cut branches longer than the level mean
    (strictly) after ceil(len/2) compartments; the mean over the whole batch,
    or (local) over each cell's own branches on the level."""
    level = 0
    while True:
        lens = [b[1] for bs in cells for b in bs if b[3] == level]
        if not lens:
            return cells
        global_mean = float(np.sum(np.array(lens, np.float64))) / len(lens)
        new_cells = []
        for bs in cells:
            mean = global_mean
            if local:
                own = [b[1] for b in bs if b[3] == level]
                if not own:
                    new_cells.append(bs)
                    continue
                mean = float(np.sum(np.array(own, np.float64))) / len(own)
            out, prox, dist = [], {}, {}
            for j, b in enumerate(bs):
                prox[j] = len(out)
                if b[3] == level and b[1] > mean and b[1] >= 2:
                    k = (b[1] + 1) // 2
                    out.append([b[0], k, b[2], b[3]])
                    dist[j] = len(out)
                    out.append([b[0] + k, b[1] - k, ("prox", j), b[3] + 1])
                else:
                    dist[j] = prox[j]
                    out.append(list(b))
            for b in out:
                if isinstance(b[2], tuple):
                    b[2] = prox[b[2][1]]
                elif b[2] >= 0:
                    b[2] = dist[b[2]]
            for b in out:
                b[3] = 0 if b[2] < 0 else out[b[2]][3] + 1
            new_cells.append(out)
        cells = new_cells
        level += 1


CAP, LANES, ALIGN = 16, 32, 8


def py_cap(bs, base, even=False, cap=CAP):
    """Branches longer than cap become chained pieces: from the proximal end,
    each piece reaches the farthest multiple of ALIGN (global natural index,
    the cell starting at `base`) within cap compartments, or the branch end.
    even: ceil(len/cap) near-equal pieces instead, the first len % pieces one
    longer."""
    out, last = [], {}
    for j, b in enumerate(bs):
        parent = -1 if b[2] < 0 else last[b[2]]
        start, end = b[0], b[0] + b[1]
        pieces = -(-b[1] // cap)
        plen, rem = divmod(b[1], pieces)
        k = 0
        while start < end:
            stop = min(end, start + cap)
            if even:
                stop = start + plen + (1 if k < rem else 0)
                k += 1
            elif stop < end:
                down = stop - (base + stop) % ALIGN
                if down > start:
                    stop = down
            out.append([start, stop - start, parent, 0 if parent < 0 else out[parent][3] + 1])
            parent = len(out) - 1
            start = stop
        last[j] = parent
    return out


UNIT_MAX = 4096


def py_units(ncomp, cells_flat):
    """Units: a cell of at most UNIT_MAX compartments; or the top part of a
    larger cell (branches whose subtree holds more than UNIT_MAX compartments)
    and one unit per remaining branch whose parent is in the top part.
    cells_flat: list per cell of global branch ids with (len, parent, level)."""
    units = []  # [kind, cell, root, [ids]]
    for c, ids in enumerate(cells_flat):
        if not ids:
            continue
        if ncomp[c] <= UNIT_MAX:
            units.append([0, c, ids[0], list(ids)])
            continue
        sub = {}
        for b in reversed(ids):
            sub[b] = sub.get(b, 0) + G["len"][b]
            pb = G["parent"][b]
            if pb >= 0:
                sub[pb] = sub.get(pb, 0) + sub[b]
        top = [b for b in ids if sub[b] > UNIT_MAX]
        topset = set(top)
        units.append([2, c, top[0], top])
        owner = {}
        for b in ids:
            if b in topset:
                continue
            pb = G["parent"][b]
            if pb in topset:
                units.append([1, c, b, [b]])
                owner[b] = len(units) - 1
            else:
                owner[b] = owner[pb]
                units[owner[b]][3].append(b)
    return units


def py_tasks(ncomp, units, sort_by_length, pack=24576, width=32, pack_whole=None):
    rl = {}
    for kind, c, root, ids in units:
        for b in ids:
            rl[b] = G["level"][b] - G["level"][root]
    tasks = []
    pack_subtrees = pack
    for kind in (0, 1, 2):
        pack = pack_whole if (kind == 0 and pack_whole is not None) else pack_subtrees
        us = [u for u in units if u[0] == kind]
        if kind == 1:  # subtrees packed per cell
            us.sort(key=lambda u: (u[1], -sum(G["len"][b] for b in u[3]), u[2]))
        else:
            us.sort(key=lambda u: (-sum(G["len"][b] for b in u[3]), u[1], u[2]))
        groups, cnt, gsize = [], [], 0
        for u in us:
            cc = np.bincount([rl[b] for b in u[3]])
            usize = sum(G["len"][b] for b in u[3])
            if kind == 2 or (kind == 1 and groups and groups[-1][0][1] != u[1]):
                fits = False  # a top part alone; subtrees of one cell per task
            elif pack < 0:  # Section 4's rule: every level at most a chunk's width of branches
                fits = bool(groups) and all((cnt[l] if l < len(cnt) else 0) + cc[l] <= width for l in range(len(cc)))
            else:
                fits = bool(groups) and gsize + usize <= pack
            if not fits:
                groups.append([])
                cnt = []
                gsize = 0
            gsize += usize
            groups[-1].append(u)
            cnt = [(cnt[l] if l < len(cnt) else 0) + (cc[l] if l < len(cc) else 0) for l in range(max(len(cnt), len(cc)))]
        for g in groups:
            ids = [b for u in g for b in u[3]]
            tasks.append((kind, py_hu(ids, rl, sort_by_length, width)))
    return tasks


def py_hu(ids, rl, sort_by_length, width):
    """Hu's list schedule of a task's dependency forest: chunks of at most
    `width` ready branches (all children in the task in earlier chunks),
    farthest from the unit root first; each chunk then ordered by length,
    longest first (stable); positions list the chunks root-side first."""
    inset = set(ids)
    pend = dict.fromkeys(ids, 0)
    for b in ids:
        if G["parent"][b] in inset:
            pend[G["parent"][b]] += 1

    def key(b):
        return (-rl[b], -G["len"][b] if sort_by_length else 0, G["cell"][b], b)

    heap = [key(b) for b in ids if pend[b] == 0]
    heapq.heapify(heap)
    chunks = []
    while heap:
        ch = [heapq.heappop(heap)[-1] for _ in range(min(width, len(heap)))]
        for b in ch:
            p = G["parent"][b]
            if p in inset:
                pend[p] -= 1
                if pend[p] == 0:
                    heapq.heappush(heap, key(p))
        ch.sort(key=lambda b: -G["len"][b])  # stable
        chunks.append(ch)
    G.setdefault("chunks", []).extend(list(reversed(chunks)))
    return [b for ch in reversed(chunks) for b in ch]


G = {}


def py_plan(ncomp, parent, split=False, sort_by_length=False, pack=0, per_lane=1, even=False, pack_whole=0):
    off = np.concatenate(([0], np.cumsum(ncomp))).astype(np.int64)
    cells = [py_branches(parent[off[c]:off[c + 1]]) for c in range(len(ncomp))]
    if split:
        cells = py_split(cells, local=split == 2)
    cells = [py_cap(bs, int(off[c]), even) for c, bs in enumerate(cells)]
    first, length, pbr, level, cell, order = [], [], [], [], [], []
    base = 0
    for c, bs in enumerate(cells):
        for b in bs:
            first.append(off[c] + b[0])
            length.append(b[1])
            pbr.append(-1 if b[2] < 0 else base + b[2])
            level.append(b[3])
            cell.append(c)
        ids = list(range(base, base + len(bs)))
        ids.sort(key=lambda g: (level[g], -length[g], g))
        order += ids
        base += len(bs)
    out = {k: np.array(v, np.int64) for k, v in
           dict(first=first, len=length, parent_branch=pbr, level=level, cell=cell, order=order).items()}
    G.clear()
    G.update(len=length, parent=pbr, level=level, cell=cell, chunks=[])
    base_of = np.concatenate(([0], np.cumsum([len(bs) for bs in cells]))).astype(np.int64)
    cells_flat = [list(range(base_of[c], base_of[c + 1])) for c in range(len(cells))]
    units = py_units(list(ncomp), cells_flat)
    default = min(24576, max(1, -(-int(np.sum(ncomp)) // 2048)))  # smaller for small batches
    whole = pack_whole if pack_whole != 0 else pack
    pack = default if pack == 0 else pack
    whole = default if whole == 0 else whole
    tasks = py_tasks(list(ncomp), units, sort_by_length, pack, LANES * per_lane, whole)
    nb = len(first)
    branch_task = np.full(nb, -1, np.int64)
    branch_kind = np.zeros(nb, np.int64)
    for kind, c, root, ids in units:
        branch_kind[ids] = kind
    torder = []
    for t, (kind, ids) in enumerate(tasks):
        branch_task[ids] = t
        torder += ids
    out["branch_task"] = branch_task
    out["branch_kind"] = branch_kind
    out["task_order"] = np.array(torder, np.int64)
    out["n_tasks"] = len(tasks)
    return out


def _compare(ncomp, parent, split, sort_by_length=False, pack=0, per_lane=1, even=False, pack_whole=0):
    plan = H.Plan(ncomp, parent, split_branches=split, host_only=True, sort_by_length=sort_by_length,
                  pack_compartments=pack, pieces_per_lane=per_lane, even_cuts=even, pack_whole=pack_whole)
    got = plan.export()
    got.update(plan.export_tasks())
    ref = py_plan(np.asarray(ncomp), np.asarray(parent), split, sort_by_length, pack, per_lane, even, pack_whole)
    assert plan.n_tasks == ref.pop("n_tasks")
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    assert got["len"].max(initial=0) <= CAP
    assert plan.n_unknowns == int(np.sum(ncomp))
    slots = plan.export_packed()
    assert plan.n_packed == slots.size
    assert np.array_equal(slots, py_packed(got, per_lane))
    return got


def py_packed(ex, per_lane):
    """Restatement of the solver layout: one block per chunk of the schedule
    (chunks in position order).  Lane j of a chunk owns its branches
    per_lane*j .. per_lane*j + per_lane - 1 and spans as many rows as its first
    (longest) branch has compartments; the lane's branches are aligned at their
    proximal ends.  Row r lists, for every lane spanning more than r rows, one
    slot per owned branch: the compartment r rows from the lane's distal start
    (r-th from the distal end of the longest; the same distance from the
    proximal end for the other), or padding (-1).  Blocks padded to multiples
    of 4 slots."""
    ln, first = ex["len"], ex["first"]
    slots = []
    for chunk in G["chunks"]:
        lanes = [chunk[k:k + per_lane] for k in range(0, len(chunk), per_lane)]
        e = 0
        for r in range(CAP):
            for own in lanes:
                rows = ln[own[0]]
                if rows <= r:
                    continue
                for h in range(per_lane):
                    t = rows - 1 - r  # distance from the proximal end
                    if h < len(own) and t < ln[own[h]]:
                        slots.append(first[own[h]] + t)
                    else:
                        slots.append(-1)
                    e += 1
        slots += [-1] * (-e % 4)
    return np.array(slots, np.int64)


def test_solver_layout_is_a_permutation():
    rng = np.random.default_rng(5)
    trees = list(tree_zoo(rng, 700).values())
    ncomp = [t.size for t in trees]
    plan = H.Plan(ncomp, np.concatenate(trees), host_only=True)
    s = plan.export_packed()
    real = s[s >= 0]
    assert np.array_equal(np.sort(real), np.arange(plan.n_unknowns))
    assert plan.n_packed - plan.n_unknowns == np.count_nonzero(s < 0)
    assert plan.n_packed % 4 == 0


@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("sort_by_length", [False, True])
@pytest.mark.parametrize("pack", [0, -1, 700])
@pytest.mark.parametrize("per_lane", [1, 2])
@pytest.mark.parametrize("even", [False, True])
def test_zoo_matches_restatement(split, sort_by_length, pack, per_lane, even):
    rng = np.random.default_rng(21)
    trees = []
    for n in (1, 2, 5, 33, 250, 5000):
        trees += list(tree_zoo(rng, n).values())
    ncomp = [t.size for t in trees]
    _compare(ncomp, np.concatenate(trees), split, sort_by_length, pack, per_lane, even)


@pytest.mark.parametrize("pack,pack_whole", [(0, 0), (9000, 3000), (-1, 5000), (12000, -1)])
def test_size_class_packing_matches_restatement(pack, pack_whole):
    w = I.WORKLOADS["uneven_steps"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:30], np.nonzero(cls == 1)[0][:3]])
    ncomp, parent = I.population_trees(w, cells)
    _compare(ncomp, parent, 0, pack=pack, pack_whole=pack_whole)


@pytest.mark.parametrize("name", ["fp64_small", "fp64_uniform", "uneven_steps", "adjoint"])
@pytest.mark.parametrize("split", [0, 1, 2])
def test_workload_samples_match_restatement(name, split):
    w = I.WORKLOADS[name]
    cells = np.arange(min(w.n_cells, 24))
    if name == "uneven_steps":  # make sure large cells are included
        cls = I.cell_classes(w)
        cells = np.concatenate([np.nonzero(cls == 0)[0][:8], np.nonzero(cls == 1)[0][:3]])
    ncomp, parent = I.population_trees(w, cells)
    got = _compare(ncomp, parent, split)
    # structure: children come after parents, every cell has one root branch
    pb = got["parent_branch"]
    assert (pb < np.arange(pb.size)).all()
    assert ((pb < 0).sum()) == len(cells)


def test_branches_cover_compartments_and_backward_order_is_valid():
    rng = np.random.default_rng(22)
    trees = [I.random_chainy_tree(rng, int(m)) for m in rng.integers(1, 400, 30)]
    ncomp = np.array([t.size for t in trees])
    parent = np.concatenate(trees)
    for split in (False, True):
        e = H.Plan(ncomp, parent, split_branches=split, host_only=True).export()
        # every compartment in exactly one branch, branches are parent chains
        cover = np.zeros(parent.size, int)
        off = np.concatenate(([0], np.cumsum(ncomp)))
        for f, l, c in zip(e["first"], e["len"], e["cell"]):
            cover[f:f + l] += 1
            loc = np.arange(f, f + l) - off[c]
            assert (parent[f + 1:f + l] == loc[:-1]).all()
        assert (cover == 1).all()
        # the proximal compartment's parent is the last compartment of the parent branch
        for b in range(e["first"].size):
            pbid = e["parent_branch"][b]
            if pbid >= 0:
                assert parent[e["first"][b]] + off[e["cell"][b]] == e["first"][pbid] + e["len"][pbid] - 1
        # reversed processing order (deepest level first) visits children before parents
        pos = np.empty_like(e["order"])
        pos[e["order"]] = np.arange(pos.size)
        has = e["parent_branch"] >= 0
        assert (pos[e["parent_branch"][has]] < pos[np.nonzero(has)[0]]).all()


def test_split_shortens_long_branches():
    rng = np.random.default_rng(23)
    w = I.WORKLOADS["fp64_uniform"]
    ncomp, parent = I.population_trees(w, np.arange(8))
    a = H.Plan(ncomp, parent, split_branches=False, host_only=True)
    b = H.Plan(ncomp, parent, split_branches=True, host_only=True)
    ea, eb = a.export(), b.export()
    # (the piece count can go either way: the cap cuts at aligned indices,
    # and a midpoint split can leave fewer aligned pieces than it adds)
    assert eb["len"].max() <= ea["len"].max()
    assert b.max_levels > a.max_levels


def test_tasks_respect_lane_rule_and_cover_branches():
    w = I.WORKLOADS["uneven_steps"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:40], np.nonzero(cls == 1)[0][:2]])
    ncomp, parent = I.population_trees(w, cells)
    plan = H.Plan(ncomp, parent, host_only=True)
    e = plan.export()
    t = plan.export_tasks()
    assert (t["branch_task"] >= 0).all()
    assert sorted(t["task_order"].tolist()) == list(range(plan.n_branches))
    # large cells are cut: top parts and subtrees; no subtree unit exceeds 4096 compartments
    assert set(np.unique(t["branch_kind"]).tolist()) == {0, 1, 2}
    # every task level (relative to unit roots) holds at most 32 branches
    pb = e["parent_branch"]
    kind = t["branch_kind"]
    root = np.arange(pb.size)
    for b in range(pb.size):  # unit root: climb while the parent is in the same unit
        r = b
        while pb[r] >= 0 and (kind[b] != 1 or kind[pb[r]] == 1):
            r = pb[r]
        root[b] = r
    rl = e["level"] - e["level"][root]
    for task in range(plan.n_tasks):
        sel = t["branch_task"] == task
        assert sel.sum() > 0


@pytest.mark.parametrize("reroot", [False, True])
def test_planner_time_is_linear(reroot):
    """Section 6: the setup work, balancing included, is linear in the number
    of cells."""
    import time
    w = I.WORKLOADS["fp64_uniform"]
    ncomp, parent = I.population_trees(w, np.arange(64))
    t = []
    for rep in (1, 8):
        nc = np.tile(ncomp, rep)
        pa = np.tile(parent, rep)
        t0 = time.perf_counter()
        for _ in range(3):
            H.Plan(nc, pa, split_branches=True, host_only=True, reroot=reroot)
        t.append((time.perf_counter() - t0) / 3)
    assert t[1] < 8 * t[0] * 2.5  # linear within noise


def test_invalid_inputs():
    with pytest.raises(H.HinesError) as e:
        H.Plan([3], np.array([-1, 0, 2], np.int32), host_only=True)
    assert e.value.code == H.HINES_ERR_NOT_HINES_ORDER
    with pytest.raises(H.HinesError) as e:
        H.Plan([2], np.array([0, 0], np.int32), host_only=True)
    assert e.value.code == H.HINES_ERR_NOT_HINES_ORDER
    with pytest.raises(H.HinesError) as e:
        H.Plan([-1], np.array([], np.int32), host_only=True)
    assert e.value.code == H.HINES_ERR_INVALID_ARG
    # empty batch and empty cells are fine
    p = H.Plan([], np.array([], np.int32), host_only=True)
    assert p.n_cells == 0 and p.n_branches == 0
    p = H.Plan([0, 3, 0], np.array([-1, 0, 1], np.int32), host_only=True)
    assert p.n_branches == 1 and list(p.offsets) == [0, 0, 3, 3]
