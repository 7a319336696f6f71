"""Benchmark of the batched Hines solver on one GB300 (one JSON line).

Step = one solve of the whole uneven population (8192 cells, 70% small / 30%
large, about 228M compartments) from FP32 d, u, b to an FP64 solution x with
the compensated FP32 elimination (hines_solve_compensated: double-float
arithmetic built from FP32 error-free transformations, no FP64 instruction),
inputs resident in HBM.  The same batch is also solved in plain FP64
(hines_solve) and with FP32 elimination + iterative refinement whose
residual is formed to FP64 accuracy from error-free FP32 products
(hines_solve_refine), for the comparison the metric asks for; each result is
checked against the oracle on sampled cells.  The inputs (2.7 GB FP32 plus
the 1.8 GB solution) exceed L2, so no flush is needed.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own replica of the population
(weak scaling, no collective on the data path); with --shard the ranks split
the population's cells instead (strong scaling).  Rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per compartment (compulsory traffic of one solve):
#   FP32 inputs, FP64 solution: read d, u, b in FP32 (12 B) + write x in FP64 (8 B)
#   FP64:                       read d, u, b in FP64 (24 B) + write x in FP64 (8 B)
BYTES_F32_IN = 20
BYTES_F64 = 32
#   passive-cable step: read s, g, u, V (32 B) + write V (8 B), FP64
BYTES_CABLE = 40


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven_mixed")
    ap.add_argument("--margin", type=float, default=0.1)
    ap.add_argument("--refine-steps", type=int, default=2)
    ap.add_argument("--cells", type=int, default=0, help="use only the first N cells (small cases, profiling)")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--refine-reps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-pieces", type=int, default=16,
                    help="cell ranges the end-to-end run pipelines its transfers over")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun, split the population's cells over the ranks (longest-processing-time "
                         "rule on compartments; strong scaling) instead of a replica per rank (weak scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (64-cell, 16384-cell, margin sweep, adjoint)")
    ap.add_argument("--cable-steps", type=int, default=1000,
                    help="passive-cable steps per captured graph for the time-stepping figure (0: skip)")
    ap.add_argument("--per-lane", type=int, default=0, choices=[0, 1, 2],
                    help="branch pieces per warp lane of every plan (0: the tuned or default options)")
    ap.add_argument("--untuned", action="store_true",
                    help="build every plan with the default options instead of the tuned ones")
    ap.add_argument("--only", choices=["headline", "solver_layout", "fp64", "cable"],
                    help="run only this solve, warmup + steps times, and print its time (small profiling runs)")
    return ap.parse_args()


def reduce_max(v: float, world: int, device: str) -> float:
    """Largest v over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, steps: int, world: int, ms_total_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * steps * world / (ms_total_max * 1e-3)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def traffic_record(kernel):
    """ncu DRAM bytes per compartment for `kernel`, if captured on the current
    sources of the task kernels (their code, the planner and the launches)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        from paper_1810_12742_gb300 import _build
        with open(path) as f:
            rec = json.load(f).get(kernel)
        if rec and rec.get("source_digest") == _build.unit_kernel_digest():
            return float(rec["dram_bytes_per_unknown"])
    except Exception:
        pass
    return None


def cpu_baseline(pop, widen, budget_s=12.0):
    """The oracle as it stands, on the host cores: repeated full-batch solves
    until about budget_s seconds of wall time."""
    import oracle
    nthreads = os.cpu_count() or 1
    d, u, b = ((pop[k].astype(np.float32).astype(np.float64) if widen else pop[k]) for k in ("d", "u", "b"))
    oracle.solve_batch(pop["ncomp"][:4], pop["parent"][:int(pop["offsets"][4])], d, u, b, nthreads)  # load
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.solve_batch(pop["ncomp"], pop["parent"], d, u, b, nthreads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    n = int(pop["offsets"][-1])
    return {"value": n * reps / el, "unit": "compartments/s", "cores": nthreads, "kind": "oracle",
            "sample": f"{reps} x the full batch ({n} compartments), serial FP64 Hines solve per cell, "
                      f"OpenMP over cells"}


def _timed_ms(torch, stream, fn, reps, warm=3):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        fn()
    a1.record(stream)
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / reps


def _cell_err(x, ref, off, cells):
    e = 0.0
    for j, c in enumerate(cells):
        sl = slice(off[c], off[c + 1])
        if off[c + 1] > off[c]:
            e = max(e, float(np.abs(x[sl] - ref[j]).max() / np.abs(ref[j]).max()))
    return e


def other_configs(torch, H, oracle, stream, max_over_ranks):
    """The other workloads, each on the GPU against the oracle: the 64-cell
    FP64 solve (latency), the 16384-cell FP64 batch, the leak-margin sweep of
    the FP32-input solves on a subset of the uneven population, and the
    200-step adjoint."""
    from paper_1810_12742_gb300 import inputs as I
    from paper_1810_12742_gb300 import rollout as R
    out = {}
    peak = load_peaks()[0]
    nth = os.cpu_count() or 1

    def oracle_cells(pop, cells, widen=False):
        off = pop["offsets"]
        refs = []
        for c in cells:
            sl = slice(off[c], off[c + 1])
            arrs = [pop[k][sl].astype(np.float32).astype(np.float64) if widen else pop[k][sl]
                    for k in ("d", "u", "b")]
            refs.append(oracle.solve_batch(pop["ncomp"][c:c + 1], pop["parent"][sl], *arrs))
        return refs

    from paper_1810_12742_gb300 import autotune as AT

    def tuned(pop, solve, layout, **extra):
        """A plan with the cached tuned options of this morphology (defaults on a miss)."""
        opts = dict(AT.cached_options(pop["ncomp"], pop["parent"], solve, layout) or {}, **extra)
        return H.Plan(pop["ncomp"], pop["parent"], **opts), opts

    # 64 binary cells x 248 compartments, FP64: launch/latency bound
    pop = I.population("fp64_small")
    plan, opts_small = tuned(pop, "f64", "natural")
    d, u, b = (torch.as_tensor(pop[k]).cuda() for k in ("d", "u", "b"))
    x = b.clone()
    us = max_over_ranks(_timed_ms(torch, stream, lambda: H.solve(plan, d, u, x), 200) * 1e3)
    x = b.clone()
    H.solve(plan, d, u, x)
    cells = np.arange(pop["ncomp"].size)
    out["fp64_small"] = {"us_per_solve": us, "compartments": int(pop["offsets"][-1]), "plan_options": opts_small,
                         "max_rel_err": _cell_err(x.cpu().numpy(), oracle_cells(pop, cells), pop["offsets"], cells)}
    # solver layout, tuned, and re-rooted at the centres (Section 6): the
    # critical path of a warp is the depth of its cells
    plan_sl, opts_sl = tuned(pop, "f64", "solver")
    out["fp64_small"]["plan_options_solver_layout"] = opts_sl
    for tag, pl in (("solver_layout", plan_sl), ("rerooted", H.Plan(pop["ncomp"], pop["parent"], reroot=True))):
        dp, up_, xp = H.pack(pl, d), H.pack_coupling(pl, u), H.pack(pl, b)
        xs = xp.clone()
        us_t = max_over_ranks(_timed_ms(torch, stream, lambda: H.solve_packed(pl, dp, up_, xs), 200) * 1e3)
        xs = xp.clone()
        H.solve_packed(pl, dp, up_, xs)
        out["fp64_small"][f"us_per_solve_{tag}"] = us_t
        out["fp64_small"][f"max_rel_err_{tag}"] = _cell_err(H.unpack(pl, xs).cpu().numpy(), oracle_cells(pop, cells),
                                                            pop["offsets"], cells)
    del plan

    # 16384 cells, about 59M compartments, FP64
    pop = I.population("fp64_uniform")
    n1 = int(pop["offsets"][-1])
    plan, opts_uni = tuned(pop, "f64", "natural")
    d, u, b = (torch.as_tensor(pop[k]).cuda() for k in ("d", "u", "b"))
    x = b.clone()
    ms = max_over_ranks(_timed_ms(torch, stream, lambda: H.solve(plan, d, u, x), 10))
    x = b.clone()
    H.solve(plan, d, u, x)
    cells = np.sort(np.random.default_rng(2).choice(pop["ncomp"].size, 32, replace=False))
    out["fp64_uniform"] = {"ms_per_solve": ms, "compartments": n1, "compartments_per_s": n1 / (ms * 1e-3),
                           "plan_options": opts_uni,
                           "hbm_frac_32B": 32 * n1 / (ms * 1e-3) / 1e9 / peak,
                           "max_rel_err": _cell_err(x.cpu().numpy(), oracle_cells(pop, cells), pop["offsets"], cells)}
    del plan, d, u, b, x, pop

    # leak-margin sweep, FP32 inputs: 256 cells of the uneven population (both classes)
    w = I.WORKLOADS["uneven_mixed"]
    cls = I.cell_classes(w)
    sub = np.concatenate([np.nonzero(cls == 0)[0][:180], np.nonzero(cls == 1)[0][:76]])
    sweep = {}
    for m in I.MARGINS:
        pop = I.population(w, cells=sub, margin=m)
        plan = H.Plan(pop["ncomp"], pop["parent"])
        f32 = {k: torch.as_tensor(pop[k].astype(np.float32)).cuda() for k in ("d", "u", "b")}
        cells = np.arange(sub.size)
        refs = oracle_cells(pop, cells, widen=True)
        wd = {k: pop[k].astype(np.float32).astype(np.float64) for k in ("d", "u")}
        cond = oracle.skeel_batch(pop["ncomp"], pop["parent"], wd["d"], wd["u"], np.concatenate(refs), nth)
        xc = H.solve_compensated(plan, f32["d"], f32["u"], f32["b"]).cpu().numpy()
        xf = f32["b"].clone()
        H.solve(plan, f32["d"], f32["u"], xf)
        r = {"skeel_cond_max": float(cond.max()),
             "compensated": _cell_err(xc, refs, pop["offsets"], cells),
             "fp32": _cell_err(xf.double().cpu().numpy(), refs, pop["offsets"], cells)}
        for st in (1, 2, 3, 4):
            xr = H.solve_refine(plan, f32["d"], f32["u"], f32["b"], steps=st).cpu().numpy()
            r[f"fp32_refine_{st}"] = _cell_err(xr, refs, pop["offsets"], cells)
        sweep[f"{m:g}"] = r
        del plan, f32
    out["margin_sweep"] = {"cells": int(sub.size), "max_rel_err": sweep}

    # branching-probability sweep (the Fig. 7.2 experiment, on 16384-cell-shaped
    # cells): the warp-task FP64 solve against the one-thread-per-cell serial
    # solve (hines_solve_f64_noalloc: one serial tree solve per thread), same data
    import ctypes
    import dataclasses
    base = I.WORKLOADS["fp64_uniform"]
    sweep_b = {}
    for ps in (0.3, 0.5, 0.9):
        wb = dataclasses.replace(base, name=f"fp64_uniform p_split {ps}", n_cells=480,
                                 classes=(dataclasses.replace(base.classes[0], p_split=ps),))
        pop = I.population(wb)
        nb_ = int(pop["offsets"][-1])
        plan = H.Plan(pop["ncomp"], pop["parent"])
        d, u, b = (torch.as_tensor(pop[k]).cuda() for k in ("d", "u", "b"))
        off_d = torch.as_tensor(pop["offsets"]).cuda()
        par_d = torch.as_tensor(pop["parent"].astype(np.int32)).cuda()
        x1, x2 = b.clone(), b.clone()
        vp = ctypes.c_void_p

        def one_thread_per_cell():
            code = H.lib().hines_solve_f64_noalloc(nb_, int(pop["ncomp"].size), vp(off_d.data_ptr()),
                                                   vp(par_d.data_ptr()), vp(d.data_ptr()), vp(u.data_ptr()),
                                                   vp(x2.data_ptr()), vp(stream.cuda_stream))
            assert code == 0
        ms_w = max_over_ranks(_timed_ms(torch, stream, lambda: H.solve(plan, d, u, x1), 20))
        ms_t = max_over_ranks(_timed_ms(torch, stream, one_thread_per_cell, 5))
        x1.copy_(b)
        x2.copy_(b)
        H.solve(plan, d, u, x1)
        one_thread_per_cell()
        same = float((x1 - x2).abs().max().item() / x2.abs().max().item())
        sweep_b[f"{ps:g}"] = {"compartments": nb_, "warp_tasks_ms": ms_w, "one_thread_per_cell_ms": ms_t,
                              "speedup": ms_t / ms_w, "max_rel_diff": same}
        del plan
    out["branching_sweep"] = sweep_b

    # adjoint: 256 cells, 200 implicit-Euler steps, checkpoints every 20
    w = I.WORKLOADS["adjoint"]
    pop = I.population(w, keys=("s", "a", "u", "g", "V0", "target"))
    plan, opts_adj = tuned(pop, "cable", "natural")
    tt = {k: torch.as_tensor(pop[k]).cuda() for k in ("s", "a", "g", "V0", "target")}

    def rollout_once():
        ga_ = tt["g"].clone().requires_grad_(True)
        aa_ = tt["a"].clone().requires_grad_(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        L_ = R.CableRollout.apply(ga_, aa_, plan, tt["s"], tt["V0"], tt["target"], w.steps, w.dt, w.E, 1,
                                  w.checkpoint_every)
        ev[1].record(stream)
        L_.backward()
        ev[2].record(stream)
        torch.cuda.synchronize()
        return L_, ga_, aa_, ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    t0 = time.perf_counter()
    rollout_once()  # builds and captures the forward and reverse graphs
    build_s = time.perf_counter() - t0
    rollout_once()
    runs = [rollout_once() for _ in range(5)]
    L, ga, aa = runs[-1][:3]
    fwd_ms = max_over_ranks(float(np.median([r[3] for r in runs])))
    bwd_ms = max_over_ranks(float(np.median([r[4] for r in runs])))
    loss, rg, ra = oracle.adjoint_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"],
                                        pop["target"], w.steps, w.dt, w.E, 1, nthreads=nth)
    gg, gaa = ga.grad.cpu().numpy(), aa.grad.cpu().numpy()
    roots = pop["offsets"][:-1]
    mask = np.ones(gaa.size, bool)
    mask[roots] = False
    out["adjoint"] = {"steps": w.steps, "compartments": int(pop["offsets"][-1]), "plan_options": opts_adj,
                      "forward_ms": fwd_ms, "backward_ms": bwd_ms, "repeats": len(runs),
                      "timing": "median of 5 after 2 warm-up rollouts (CUDA events); the first rollout builds "
                                "and captures the forward and reverse graphs",
                      "graph_build_s": build_s,
                      "loss_rel_err": abs(L.item() - float(loss.sum())) / abs(float(loss.sum())),
                      "grad_g_rel_err": float(np.abs(gg - rg).max() / np.abs(rg).max()),
                      "grad_a_rel_err": float(np.abs(gaa[mask] - ra[mask]).max() / np.abs(ra[mask]).max())}
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1810_12742_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    cells = np.arange(args.cells) if args.cells else None
    sharded = args.shard and world > 1 and args.impl != "reference"
    if sharded:  # every rank computes the same split; nothing is exchanged
        from paper_1810_12742_gb300 import shard as S
        nc_all, _ = I.population_trees(w, cells)
        part = S.lpt_partition(nc_all, world)[rank]
        cells = part if cells is None else cells[part]
    pop = I.population(w, cells=cells, margin=args.margin)
    n = int(pop["offsets"][-1])
    n_job = int(nc_all.sum()) if sharded else n * world  # compartments the whole job solves per step
    widen = True
    config = {"workload": w.name, "cells": int(pop["ncomp"].size), "compartments": n,
              "leak_margin": args.margin, "path": "hines_solve_compensated: FP32 d, u, b -> FP64 x, "
              "double-float elimination from FP32 error-free transformations",
              "l2": "inputs and solution (4.6 GB at full size) exceed L2; no flush",
              "seed": f"numpy PCG64 per cell, base {I.SEED_BASE}",
              "parallelism": (f"cells split over {world} ranks (longest-processing-time rule on compartments)"
                              if sharded else f"{world} replica(s), one per GPU, no collective on the data path")}
    if sharded:
        config["job_compartments"] = n_job
    metric = "compartments solved/sec per GB300 and % of HBM roofline, FP32+refine vs FP64"

    if args.impl == "reference":
        # the oracle as it stands on the host cores: a step is one solve of the
        # whole batch (FP64 Listing 2 per cell, OpenMP over cells), warmup
        # untimed steps, then steps timed steps
        if rank != 0:
            return
        import oracle
        nthreads = os.cpu_count() or 1
        d, u, b = (pop[k].astype(np.float32).astype(np.float64) for k in ("d", "u", "b"))
        for _ in range(args.warmup):
            oracle.solve_batch(pop["ncomp"], pop["parent"], d, u, b, nthreads)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.solve_batch(pop["ncomp"], pop["parent"], d, u, b, nthreads)
        el = time.perf_counter() - t0
        value = n * args.steps / el
        cb = {"value": value, "unit": "compartments/s", "cores": nthreads, "kind": "oracle",
              "sample": f"each step one solve of the whole batch ({n} compartments): serial FP64 Hines solve "
                        f"per cell, OpenMP over cells; {args.steps} timed steps after {args.warmup} warm-up"}
        line = {"impl": "reference", "metric": metric, "value": value, "unit": "compartments/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config, "cpu_baseline": cb,
                "e2e": {"value": value, "unit": "compartments/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1810_12742_gb300 import hines as H

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        return reduce_max(v, world, "cuda")

    # Each solve runs on the plan options the autotuner chose for this
    # morphology on a GB300 (the cache shipped with the package; nothing is
    # tuned here).  A cache miss, --untuned or --per-lane: default options.
    from paper_1810_12742_gb300 import autotune as AT
    plans, plan_options = {}, {}

    def plan_for(solve, layout):
        opts = None
        if args.per_lane:
            opts = {"pieces_per_lane": args.per_lane}
        elif not args.untuned:
            opts = AT.cached_options(pop["ncomp"], pop["parent"], solve, layout)
        plan_options[f"{solve}/{layout}"] = {"options": opts or {}, "tuned": opts is not None and not args.per_lane}
        key = json.dumps(opts or {}, sort_keys=True)
        if key not in plans:
            t0 = time.perf_counter()
            plans[key] = H.Plan(pop["ncomp"], pop["parent"], **(opts or {}))
            plan_options[f"{solve}/{layout}"]["plan_create_s"] = time.perf_counter() - t0
        return plans[key]

    t_plan = time.perf_counter()
    plan = plan_for("compensated", "natural")
    config["plan_create_s"] = time.perf_counter() - t_plan  # host planner + upload, once per morphology
    config["plan_options"] = plan_options
    f32 = {k: torch.as_tensor(pop[k].astype(np.float32)).cuda() for k in ("d", "u", "b")}
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        H.solve_compensated(plan, f32["d"], f32["u"], f32["b"], x)

    if args.only:
        if args.only == "solver_layout":
            plan = plan_for("compensated", "solver")
            pk = {"d": H.pack(plan, f32["d"]), "u": H.pack_coupling(plan, f32["u"]), "b": H.pack(plan, f32["b"])}
            xpk = torch.empty(plan.n_packed, dtype=torch.float64, device="cuda")

            def step():  # noqa: F811
                H.solve_compensated_packed(plan, pk["d"], pk["u"], pk["b"], xpk)
        elif args.only == "fp64":
            plan = plan_for("f64", "natural")
            f64 = {k: torch.as_tensor(pop[k]).cuda() for k in ("d", "u", "b")}
            x64 = torch.empty_like(f64["b"])

            def step():  # noqa: F811
                x64.copy_(f64["b"])
                H.solve(plan, f64["d"], f64["u"], x64)
        elif args.only == "cable":  # one passive-cable step (rebuild fused with the FP64 solve), natural layout
            plan = plan_for("cable", "natural")
            ws = I.WORKLOADS["uneven_steps"]
            cp = I.population(ws, cells=cells, keys=("s", "u", "g", "V0"))
            cs = {k: torch.as_tensor(cp[k]).cuda() for k in ("s", "g", "u", "V0")}

            def step():  # noqa: F811
                H.cable_step(plan, cs["s"], cs["g"], cs["u"], cs["V0"], ws.dt, ws.E, 1)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"only": args.only, "compartments": n, "ms_per_step": e0.elapsed_time(e1) / args.steps,
                              "status": plan.status()}), flush=True)
        return

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    value = n_job * args.steps / (ms_total * 1e-3) if sharded else job_value(n, args.steps, world, ms_total)
    status = plan.status()

    # parity on sampled cells against the oracle
    import oracle
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(pop["ncomp"].size, min(64, pop["ncomp"].size), replace=False))
    off = pop["offsets"]

    def max_rel_err(xd, widen):
        xs = xd.cpu().numpy() if hasattr(xd, "cpu") else xd
        err = 0.0
        for c in sample:
            sl = slice(off[c], off[c + 1])
            if off[c + 1] == off[c]:
                continue
            arrs = [pop[k][sl].astype(np.float32).astype(np.float64) if widen else pop[k][sl]
                    for k in ("d", "u", "b")]
            ref = oracle.solve_batch(pop["ncomp"][c:c + 1], pop["parent"][sl], *arrs)
            err = max(err, float(np.abs(xs[sl] - ref).max() / np.abs(ref).max()))
        return err

    err = max_rel_err(x, True)

    def timed(fn, reps):
        ms = []
        for it in range(args.warmup + reps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn()
            a1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ms.append(a0.elapsed_time(a1))
        return max_over_ranks(float(np.mean(ms)))

    # FP64 solve of the same batch (in place; b is restored outside the timed events)
    plan64 = plan_for("f64", "natural")
    f64 = {k: torch.as_tensor(pop[k]).cuda() for k in ("d", "u", "b")}
    x64 = torch.empty_like(f64["b"])
    ms64 = []
    for it in range(args.warmup + args.fp64_steps):
        x64.copy_(f64["b"])
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        H.solve(plan64, f64["d"], f64["u"], x64)
        a1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            ms64.append(a0.elapsed_time(a1))
    ms64 = max_over_ranks(float(np.mean(ms64)))
    err64 = max_rel_err(x64, False)
    del f64, x64

    # FP32 elimination + residual refinement (the same FP32 inputs): the FP32
    # solve, then per step one pass that forms the residual and eliminates it
    # with the FP32 factor, and one that substitutes the correction
    xr = torch.empty(n, dtype=torch.float64, device="cuda")
    refine = {}
    plan_r = plan_for("refine", "natural")
    for st in sorted({1, args.refine_steps}):
        ms_r = timed(lambda: H.solve_refine(plan_r, f32["d"], f32["u"], f32["b"], xr, st), args.refine_reps)
        refine[st] = (ms_r, max_rel_err(xr, True))
    ms_ref, err_ref = refine[args.refine_steps]
    del xr

    # the same solve on arrays kept in the solver layout (Section 5's per-chunk
    # interleaving): what a simulation that stores its state in that layout pays
    plan_s = plan_for("compensated", "solver")
    pk = {"d": H.pack(plan_s, f32["d"]), "u": H.pack_coupling(plan_s, f32["u"]), "b": H.pack(plan_s, f32["b"])}
    xpk = torch.empty(plan_s.n_packed, dtype=torch.float64, device="cuda")
    ms_pk = timed(lambda: H.solve_compensated_packed(plan_s, pk["d"], pk["u"], pk["b"], xpk), args.steps)
    err_pk = max_rel_err(H.unpack(plan_s, xpk), True)
    ms_pack = timed(lambda: [H.pack(plan_s, f32["d"], pk["d"]), H.pack_coupling(plan_s, f32["u"], pk["u"]),
                             H.pack(plan_s, f32["b"], pk["b"])], 3)
    ms_unpack = timed(lambda: H.unpack(plan_s, xpk, x), 3)
    n_packed_s = plan_s.n_packed
    del pk, xpk

    # the same, with every cell re-rooted at its centre (Section 6): couplings
    # packed through the plan's edge map
    t_rr = time.perf_counter()
    plan_rr = H.Plan(pop["ncomp"], pop["parent"], reroot=True)
    plan_rr_s = time.perf_counter() - t_rr
    pk = {"d": H.pack(plan_rr, f32["d"]), "u": H.pack_coupling(plan_rr, f32["u"]), "b": H.pack(plan_rr, f32["b"])}
    xpk = torch.empty(plan_rr.n_packed, dtype=torch.float64, device="cuda")
    ms_rr = timed(lambda: H.solve_compensated_packed(plan_rr, pk["d"], pk["u"], pk["b"], xpk), args.steps)
    err_rr = max_rel_err(H.unpack(plan_rr, xpk), True)
    del pk, xpk, plan_rr

    # passive-cable time stepping (rebuild of d and b from V fused with the FP64
    # solve), the same trees: K steps captured in one CUDA graph, natural layout
    # and solver layout
    cable = None
    if args.cable_steps > 0:
        from paper_1810_12742_gb300 import rollout as R
        ws = I.WORKLOADS["uneven_steps"]
        cp = I.population(ws, cells=cells, keys=("s", "a", "u", "g", "V0"))
        cs = {k: torch.as_tensor(cp[k]).cuda() for k in ("s", "g", "u", "V0")}
        cable = {"steps_per_graph": args.cable_steps, "algorithmic_bytes_per_compartment": BYTES_CABLE,
                 "path": "hines_cable_step (theta 1) x steps in one CUDA graph; *_factor_reuse: the first step "
                         "full, the others hines_cable_step_reuse (constant matrix, a separate variant)"}
        for layout, reuse in (("natural", False), ("solver", False), ("natural", True), ("solver", True)):
            V = cs["V0"].clone()
            st = R.CableStepper(plan_for("cable", layout), cs["s"], cs["g"], cs["u"], V, ws.dt, ws.E, 1,
                                steps=args.cable_steps,
                                layout=layout, reuse_factor=reuse)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            st.replay()
            a1.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(a0.elapsed_time(a1) / args.cable_steps)
            Vn = st.fetch().cpu().numpy()
            err_c = 0.0
            for c in sample[:16]:
                sl = slice(off[c], off[c + 1])
                ref, _ = oracle.steps_batch(pop["ncomp"][c:c + 1], pop["parent"][sl], cp["s"][sl], cp["g"][sl],
                                            cp["a"][sl], cp["V0"][sl], args.cable_steps, ws.dt, ws.E, 1)
                err_c = max(err_c, float(np.abs(Vn[sl] - ref).max() / np.abs(ref).max()))
            cable[layout + ("_factor_reuse" if reuse else "")] = {
                "ms_per_step": ms, "compartments_per_s": n / (ms * 1e-3), "max_rel_err": err_c,
                "hbm_frac": BYTES_CABLE * n / (ms * 1e-3) / 1e9 / load_peaks()[0]}
            del st, V
        del cs, cp

    configs = None if (args.no_configs or args.cells) else other_configs(torch, H, oracle, stream, max_over_ranks)

    # end to end through the public API with pinned host buffers
    host = {k: torch.as_tensor(pop[k].astype(np.float32)).pin_memory() for k in ("d", "u", "b")}
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    pipe = H.HostPipeline(pop["ncomp"], pop["parent"], pieces=args.e2e_pieces,
                          **plan_options["compensated/natural"]["options"])
    e2e_ms = timed(lambda: pipe.solve_compensated(host["d"], host["u"], host["b"], xh), args.e2e_steps)
    e2e_err = max_rel_err(xh.numpy(), True)
    del pipe

    peak, peak_kind = load_peaks()
    achieved = BYTES_F32_IN * n / (ms_step * 1e-3) / 1e9
    kernel = "k_units<CompMode>"
    tr = traffic_record(kernel)
    tr_pk = traffic_record("k_units<CompModeT<solver layout>>")
    line = {
        "metric": metric, "value": value, "unit": "compartments/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "max_rel_err": err, "status": status,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None if tr is None else tr * n,
                     "kernel": kernel + " (the two launches of one solve)",
                     "algorithmic_bytes_per_compartment": BYTES_F32_IN,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json), of {peak_kind}"},
        "fp64": {"value": n / (ms64 * 1e-3), "unit": "compartments/s", "ms_per_solve": ms64,
                 "max_rel_err": err64, "roofline_frac": BYTES_F64 * n / (ms64 * 1e-3) / 1e9 / peak,
                 "speedup_of_compensated": ms64 / ms_step},
        "solver_layout": {"value": n / (ms_pk * 1e-3), "unit": "compartments/s", "ms_per_solve": ms_pk,
                          "traffic": None if tr_pk is None else tr_pk * n,
                          "max_rel_err": err_pk, "n_packed": n_packed_s,
                          "roofline_frac": BYTES_F32_IN * n / (ms_pk * 1e-3) / 1e9 / peak,
                          "pack_d_u_b_ms": ms_pack, "unpack_x_ms": ms_unpack,
                          "path": "hines_solve_compensated_packed on d, u, b, x kept in the solver layout",
                          "rerooted": {"ms_per_solve": ms_rr, "max_rel_err": err_rr, "plan_create_s": plan_rr_s,
                                       "path": "the same on a plan with every cell re-rooted at its centre"}},
        "cable_steps": cable,
        "configs": configs,
        "fp32_refine": {"value": n / (ms_ref * 1e-3), "unit": "compartments/s", "ms_per_solve": ms_ref,
                        "refine_steps": args.refine_steps, "max_rel_err": err_ref,
                        "roofline_frac": BYTES_F32_IN * n / (ms_ref * 1e-3) / 1e9 / peak,
                        "speedup_over_fp64": ms64 / ms_ref,
                        "steps": {str(k): {"ms_per_solve": v[0], "max_rel_err": v[1],
                                           "roofline_frac": BYTES_F32_IN * n / (v[0] * 1e-3) / 1e9 / peak}
                                  for k, v in refine.items()},
                        "path": "hines_solve_refine: FP32 solve (factor kept), then per step a residual + "
                                "correction-elimination pass and a correction-substitution pass"},
        "e2e": {"value": n_job / (e2e_ms * 1e-3), "unit": "compartments/s",
                "h2d_bytes_per_step": 12 * n_job, "d2h_bytes_per_step": 8 * n_job, "max_rel_err": e2e_err,
                "path": f"C-ABI hines_pipeline_solve_compensated (through hines.HostPipeline) on pinned host "
                        f"arrays: the batch cut into {args.e2e_pieces} runs of consecutive cells, each with its own "
                        "plan; per run the host-to-device copies, the device solve and the device-to-host copy on "
                        "three internal streams, overlapped"},
        "clocks": clk.summary(),
        "gpu_launches": 2 * args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pop, widen)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
