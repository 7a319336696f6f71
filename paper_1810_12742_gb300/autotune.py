"""Autotuner of the plan options for one morphology (orchestration only).

The planner's free choices change the schedule, and with it only the order
in which the elimination adds contributions into a compartment:

* per size class, how many compartments a warp task holds (whole cells of at
  most 4096 compartments: ``pack_whole``; the subtrees of larger cells:
  ``pack_compartments``);
* the branch-to-lane mapping (``pieces_per_lane``: one piece per lane, or two
  run at once);
* how long branches are cut (``even_cuts``: at multiples of 8 of the natural
  layout, so that pieces share no memory sector, or into near-equal pieces);
* Section 6's split at the level means, over the batch or per cell
  (``split_branches`` 1 / 2), whether ready branches of equal depth are taken
  longest first, and re-rooting at the centres (solver layout only);
* for the FP64 solves and cable steps, where the factor waits between the
  sweeps (``fp64_factor``: natural positions or the chunks' block order).

Which is fastest depends on the batch and on the solve, so ``tune_plan``
times candidates on a synthetic diagonally dominant system of the same
morphology, one option at a time from the defaults (coordinate descent: each
option's values are timed with the best of the others kept), and returns the
fastest plan.  The choice is cached, keyed by a hash of the morphology, the
solve, the layout and the device, so a morphology is tuned once; the cache
that ships with the package holds the benchmark workloads tuned on a GB300.

    python -m paper_1810_12742_gb300.autotune --workload uneven_mixed --solve compensated --layout natural
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os

import numpy as np

from . import hines as H

TUNED_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_plans.json")

# option -> values tried, in the order the search visits them
SEARCH_SPACE = (
    ("even_cuts", (False, True)),
    ("pack_compartments", (6144, 12288, 24576, 49152)),
    ("pack_whole", (0, 6144, 49152)),
    ("pieces_per_lane", (1, 2)),
    ("split_branches", (0, 1, 2)),
    ("sort_by_length", (False, True)),
)
SOLVER_LAYOUT_SPACE = (("reroot", (False, True)),)
# where the FP64 solves keep their factor (natural positions or block order)
FP64_SPACE = (("fp64_factor", (1, 2)),)
SOLVES = ("compensated", "f64", "cable", "refine")

# kept for callers that pass explicit candidate lists
DEFAULT_CANDIDATES = (
    dict(pack_compartments=12288),
    dict(pack_compartments=16384),
    dict(pack_compartments=24576),
    dict(pack_compartments=32768),
    dict(pack_compartments=24576, sort_by_length=True),
    dict(pack_compartments=24576, split_branches=True),
)
SOLVER_LAYOUT_CANDIDATES = (
    dict(pack_compartments=24576, reroot=True),
    dict(pack_compartments=32768, reroot=True),
)


def _key(ncomp, parent, solve, layout):
    import torch
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ncomp, np.int32).tobytes())
    h.update(np.ascontiguousarray(parent, np.int32).tobytes())
    h.update(f"{solve}|{layout}|{torch.cuda.get_device_name()}".encode())
    return h.hexdigest()


def _system(ncomp, parent, seed=0):
    """A synthetic system of the morphology (FP64, device): u = -a with
    a ~ U[0.5, 2] per edge, d = s + sum of a over the edges, s ~ U[0.01, 0.1],
    b ~ U[-1, 1]."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    nc = np.asarray(ncomp, np.int64)
    off = np.concatenate(([0], np.cumsum(nc)))
    n = int(off[-1])
    loc = np.asarray(parent, np.int64)
    par = np.where(loc >= 0, loc + np.repeat(off[:-1], nc), np.arange(n))  # global parent; a root points to itself
    roots = off[:-1][nc > 0]
    a = torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * 1.5 + 0.5
    a[torch.as_tensor(roots, device="cuda")] = 0.0
    s = torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * 0.09 + 0.01
    b = torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * 2.0 - 1.0
    p = torch.as_tensor(par, device="cuda")
    d = s + a
    d.index_add_(0, p, a)
    return d, -a, b


def _timer(solve, layout, plan, d, u, b):
    import torch
    if solve in ("compensated", "refine"):
        d32, u32, b32 = (t.float() for t in (d, u, b))
        if layout == "solver":
            if solve == "refine":
                raise ValueError("the refinement takes natural-layout arrays")
            pd, pu, pb = H.pack(plan, d32), H.pack_coupling(plan, u32), H.pack(plan, b32)
            px = torch.empty(plan.n_packed, dtype=torch.float64, device="cuda")
            return lambda: H.solve_compensated_packed(plan, pd, pu, pb, px)
        x = torch.empty(plan.n_unknowns, dtype=torch.float64, device="cuda")
        if solve == "refine":
            return lambda: H.solve_refine(plan, d32, u32, b32, x, 1)
        return lambda: H.solve_compensated(plan, d32, u32, b32, x)
    if solve == "f64":
        if layout == "solver":
            pd, pu, pb = H.pack(plan, d), H.pack_coupling(plan, u), H.pack(plan, b)
            return lambda: H.solve_packed(plan, pd, pu, pb)
        x = b.clone()
        return lambda: H.solve(plan, d, u, x)
    if solve == "cable":  # one passive-cable step (s, g, u; V advanced in place)
        s_ = torch.full_like(d, 0.05)
        g_ = torch.full_like(d, 0.5)
        if layout == "solver":
            ps, pg, pu, pV = H.pack(plan, s_), H.pack(plan, g_), H.pack_coupling(plan, u), H.pack(plan, b)
            return lambda: H.cable_step_packed(plan, ps, pg, pu, pV, 0.025, -65.0, 1)
        V = b.clone()
        return lambda: H.cable_step(plan, s_, g_, u, V, 0.025, -65.0, 1)
    raise ValueError(f"solve: expected one of {SOLVES}, got {solve!r}")


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _search(ncomp, parent, solve, layout, reps, d, u, b):
    """Coordinate descent over the option space from the defaults."""
    space = SEARCH_SPACE + (SOLVER_LAYOUT_SPACE if layout == "solver" else ()) + (
        FP64_SPACE if solve in ("f64", "cable") else ())
    best_opts, best_ms, best_plan = {}, None, None
    times = {}
    for name, values in space:
        for v in values:
            opts = dict(best_opts, **{name: v})
            key = json.dumps(opts, sort_keys=True)
            if key in times:
                continue
            plan = H.Plan(ncomp, parent, **opts)
            ms = _time(_timer(solve, layout, plan, d, u, b), reps)
            times[key] = ms
            if best_ms is None or ms < best_ms:
                if best_plan is not None:
                    best_plan.close()
                best_opts, best_ms, best_plan = opts, ms, plan
            else:
                plan.close()
    return best_plan, best_opts, times


def cached_options(ncomp, parent, solve: str, layout: str, cache_path: str = TUNED_CACHE):
    """The tuned options of this morphology, solve and layout from the cache,
    or None when it holds none (nothing is built or timed)."""
    if not cache_path or not os.path.exists(cache_path):
        return None
    with open(cache_path) as f:
        rec = json.load(f).get(_key(ncomp, parent, solve, layout))
    return None if rec is None else rec["options"]


def tune_plan(ncomp, parent, solve: str = "compensated", layout: str = "natural", candidates=None,
              reps: int = 3, cache_path: str | None = None, tune_on_miss: bool = True):
    """Returns (plan, report): the plan with the fastest options for this
    morphology, solve and layout, and {"options", "ms" (per candidate),
    "cached"}.  Without explicit candidates the options are searched one at a
    time from the defaults (see SEARCH_SPACE).  A plan rebuilt from cached
    options schedules exactly as the tuned one did.  tune_on_miss=False: a
    cache miss returns the default plan untuned ({"options": None})."""
    if candidates is not None:
        candidates = list(candidates)
        if layout != "solver" and any(c.get("reroot") for c in candidates):
            raise ValueError("re-rooted plans take the solver layout only")
    key = _key(ncomp, parent, solve, layout)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        opts = cache[key]["options"]
        return H.Plan(ncomp, parent, **opts), {"options": opts, "ms": cache[key]["ms"], "cached": True}
    if not tune_on_miss:
        return H.Plan(ncomp, parent), {"options": None, "ms": {}, "cached": False}
    d, u, b = _system(ncomp, parent)
    if candidates is None:
        best_plan, best_opts, times = _search(ncomp, parent, solve, layout, reps, d, u, b)
    else:
        times, best_opts, best_plan, best_ms = {}, None, None, None
        for opts in candidates:
            plan = H.Plan(ncomp, parent, **opts)
            ms = _time(_timer(solve, layout, plan, d, u, b), reps)
            times[json.dumps(opts, sort_keys=True)] = ms
            if best_ms is None or ms < best_ms:
                if best_plan is not None:
                    best_plan.close()
                best_opts, best_ms, best_plan = opts, ms, plan
            else:
                plan.close()
    report = {"options": best_opts, "ms": times, "cached": False}
    if cache_path:
        cache[key] = {"options": best_opts, "ms": times}
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return best_plan, report


def main(argv=None):
    from . import inputs as I
    ap = argparse.ArgumentParser(description="tune the plan options of a benchmark workload's morphology")
    ap.add_argument("--workload", default="uneven_mixed", choices=sorted(I.WORKLOADS))
    ap.add_argument("--solve", default="compensated", choices=SOLVES)
    ap.add_argument("--layout", default="natural", choices=("natural", "solver"))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cache", default=TUNED_CACHE)
    a = ap.parse_args(argv)
    ncomp, parent = I.population_trees(I.WORKLOADS[a.workload])
    plan, rep = tune_plan(ncomp, parent, a.solve, a.layout, reps=a.reps, cache_path=a.cache)
    print(json.dumps({"workload": a.workload, "solve": a.solve, "layout": a.layout, **rep}), flush=True)


if __name__ == "__main__":
    main()
