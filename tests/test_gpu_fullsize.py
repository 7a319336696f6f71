"""Parity at the full workload sizes, in the launch configuration bench.py
times: the whole population is solved on the GPU and EVERY cell is compared,
element by element, with the oracle's solve of the same inputs (the oracle
solves the whole batch on all host cores in well under a second).

Modes: FP64 (hines_solve), the compensated solve in both layouts, FP32
elimination with FP64 refinement, and plain FP32.  The FP32-input modes are
compared with the oracle's FP64 solve of the FP32 inputs widened exactly."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 1


def per_cell_rel_err(x, ref, off):
    """max_i |x_i - ref_i| / max_i |ref_i| over each cell's compartments."""
    nonempty = off[1:] > off[:-1]
    starts = off[:-1][nonempty]
    num = np.maximum.reduceat(np.abs(x - ref), starts)
    den = np.maximum.reduceat(np.abs(ref), starts)
    return num / np.maximum(den, 1e-300)


def _oracle(pop, widen):
    arrs = [pop[k].astype(np.float32).astype(np.float64) if widen else pop[k] for k in ("d", "u", "b")]
    return oracle.solve_batch(pop["ncomp"], pop["parent"], *arrs, NTH)


def test_uneven_population_full_size_every_cell():
    w = I.WORKLOADS["uneven_mixed"]
    pop = I.population(w, margin=0.1)
    off = pop["offsets"]
    plan = H.Plan(pop["ncomp"], pop["parent"])
    ref32 = _oracle(pop, True)
    f32 = {k: torch.as_tensor(pop[k].astype(np.float32)).cuda() for k in ("d", "u", "b")}

    xc = H.solve_compensated(plan, f32["d"], f32["u"], f32["b"]).cpu().numpy()
    assert per_cell_rel_err(xc, ref32, off).max() <= 1e-10
    pk = {k: H.pack(plan, f32[k]) for k in ("d", "u", "b")}
    xp = H.unpack(plan, H.solve_compensated_packed(plan, pk["d"], pk["u"], pk["b"])).cpu().numpy()
    assert per_cell_rel_err(xp, ref32, off).max() <= 1e-10
    del pk, xp
    xr = H.solve_refine(plan, f32["d"], f32["u"], f32["b"], steps=2).cpu().numpy()
    assert per_cell_rel_err(xr, ref32, off).max() <= 1e-10
    del xr
    xf = f32["b"].clone()
    H.solve(plan, f32["d"], f32["u"], xf)
    assert per_cell_rel_err(xf.double().cpu().numpy(), ref32, off).max() <= 1e-5
    del f32, xf, ref32

    ref64 = _oracle(pop, False)
    x64 = torch.as_tensor(pop["b"]).cuda()
    H.solve(plan, torch.as_tensor(pop["d"]).cuda(), torch.as_tensor(pop["u"]).cuda(), x64)
    assert per_cell_rel_err(x64.cpu().numpy(), ref64, off).max() <= 1e-12
    assert plan.status() == 0


def test_uniform_population_full_size_fp64_every_cell():
    w = I.WORKLOADS["fp64_uniform"]
    pop = I.population(w)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = torch.as_tensor(pop["b"]).cuda()
    H.solve(plan, torch.as_tensor(pop["d"]).cuda(), torch.as_tensor(pop["u"]).cuda(), x)
    assert per_cell_rel_err(x.cpu().numpy(), _oracle(pop, False), pop["offsets"]).max() <= 1e-12


@pytest.mark.parametrize("layout", ["natural", "solver"])
def test_cable_steps_full_size_every_cell(layout):
    """Three passive-cable steps (rebuild of d and b from V fused with the FP64
    solve) on the whole uneven population, then three more re-using the
    first step's factor (the matrix is constant), each cell against the
    oracle stepper after 3 and after 6 steps."""
    w = I.WORKLOADS["uneven_steps"]
    cp = I.population(w, keys=("s", "a", "u", "g", "V0"))
    off = cp["offsets"]
    plan = H.Plan(cp["ncomp"], cp["parent"], reroot=False)
    cs = {k: torch.as_tensor(cp[k]).cuda() for k in ("s", "g", "u", "V0")}
    solver = layout == "solver"
    if solver:
        s, g, u, V = H.pack(plan, cs["s"]), H.pack(plan, cs["g"]), H.pack_coupling(plan, cs["u"]), H.pack(plan, cs["V0"])
    else:
        s, g, u, V = cs["s"], cs["g"], cs["u"], cs["V0"].clone()
    del cs
    step = H.cable_step_packed if solver else H.cable_step
    for _ in range(3):
        step(plan, s, g, u, V, w.dt, w.E, 1)
    v3 = (H.unpack(plan, V) if solver else V).cpu().numpy()
    for _ in range(3):
        H.cable_step_reuse(plan, s, g, u, V, w.dt, w.E, 1, solver_layout=solver)
    v6 = (H.unpack(plan, V) if solver else V).cpu().numpy()
    assert plan.status() == 0
    del s, g, u, V
    ref3, _ = oracle.steps_batch(cp["ncomp"], cp["parent"], cp["s"], cp["g"], cp["a"], cp["V0"], 3, w.dt, w.E, 1, NTH)
    assert per_cell_rel_err(v3, ref3, off).max() <= 1e-12
    ref6, _ = oracle.steps_batch(cp["ncomp"], cp["parent"], cp["s"], cp["g"], cp["a"], ref3, 3, w.dt, w.E, 1, NTH)
    assert per_cell_rel_err(v6, ref6, off).max() <= 1e-12
