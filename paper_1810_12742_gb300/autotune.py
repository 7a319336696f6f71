"""Autotuner of the plan options for one morphology (orchestration only).

The planner's free choices -- how many compartments a warp task holds, whether
ready branches of equal depth are taken longest first, whether long branches
are split at their level's mean, whether cells are re-rooted at their centres
(both Section 6) -- change the schedule, and with it only the order in which
the elimination adds contributions into a compartment.  Which
is fastest depends on the batch (its size classes, depth, branching) and on the
solve, so ``tune_plan`` times each candidate on a synthetic diagonally dominant
system of the same morphology and returns the fastest plan.  The choice is
cached, keyed by a hash of the morphology, the solve, the layout and the device,
so a morphology is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import hines as H

DEFAULT_CANDIDATES = (
    dict(pack_compartments=12288),
    dict(pack_compartments=16384),
    dict(pack_compartments=24576),
    dict(pack_compartments=32768),
    dict(pack_compartments=24576, sort_by_length=True),
    dict(pack_compartments=24576, split_branches=True),
)
# re-rooted plans (Section 6) take solver-layout arrays only
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
    if solve == "compensated":
        d32, u32, b32 = (t.float() for t in (d, u, b))
        if layout == "solver":
            pd, pu, pb = H.pack(plan, d32), H.pack_coupling(plan, u32), H.pack(plan, b32)
            px = torch.empty(plan.n_packed, dtype=torch.float64, device="cuda")
            return lambda: H.solve_compensated_packed(plan, pd, pu, pb, px)
        x = torch.empty(plan.n_unknowns, dtype=torch.float64, device="cuda")
        return lambda: H.solve_compensated(plan, d32, u32, b32, x)
    if solve == "f64":
        if layout == "solver":
            pd, pu, pb = H.pack(plan, d), H.pack_coupling(plan, u), H.pack(plan, b)
            return lambda: H.solve_packed(plan, pd, pu, pb)
        x = b.clone()
        return lambda: H.solve(plan, d, u, x)
    raise ValueError(f"solve: expected 'compensated' or 'f64', got {solve!r}")


def tune_plan(ncomp, parent, solve: str = "compensated", layout: str = "natural", candidates=None,
              reps: int = 3, cache_path: str | None = None):
    """Returns (plan, report): the plan with the fastest options for this
    morphology, solve and layout, and {"options", "ms" (per candidate),
    "cached"}.  A plan rebuilt from cached options schedules exactly as the
    tuned one did."""
    import torch
    if candidates is None:
        candidates = DEFAULT_CANDIDATES + (SOLVER_LAYOUT_CANDIDATES if layout == "solver" else ())
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
    d, u, b = _system(ncomp, parent)
    times, best, best_plan = [], None, None
    for opts in candidates:
        plan = H.Plan(ncomp, parent, **opts)
        fn = _timer(solve, layout, plan, d, u, b)
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        times.append(ms)
        if best is None or ms < times[best]:
            best, best_plan = len(times) - 1, plan
        else:
            plan.close()
    report = {"options": candidates[best], "ms": dict(zip((json.dumps(c, sort_keys=True) for c in candidates), times)),
              "cached": False}
    if cache_path:
        cache[key] = {"options": candidates[best], "ms": report["ms"]}
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best_plan, report
