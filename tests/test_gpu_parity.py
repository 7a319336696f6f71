"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (relative max-norm error per cell, ||x_gpu - x_oracle||_inf /
||x_oracle||_inf): FP64 1e-12, plain FP32 1e-5 (at the default leak margin),
FP32 elimination + refinement (its residual formed to FP64 accuracy) and the
compensated solve 1e-10.  The FP32 paths are compared with
the oracle's FP64 solve of the FP32 inputs widened exactly to FP64.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I
from tests.helpers import problem, tree_zoo

pytestmark = pytest.mark.gpu

TOL_F64, TOL_F32, TOL_REFINE = 1e-12, 1e-5, 1e-10


def cell_rel_err(x, ref, off):
    errs = np.empty(len(off) - 1)
    for c in range(len(off) - 1):
        sl = slice(off[c], off[c + 1])
        if off[c + 1] == off[c]:
            errs[c] = 0.0
            continue
        errs[c] = np.abs(x[sl] - ref[sl]).max() / max(np.abs(ref[sl]).max(), 1e-300)
    return errs


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def zoo_batch(seed, sizes=(1, 2, 3, 17, 64, 65, 300, 1000)):
    rng = np.random.default_rng(seed)
    trees, coef = [], {k: [] for k in ("d", "u", "b", "s", "a")}
    for n in sizes:
        for t in tree_zoo(rng, n).values():
            trees.append(t)
            pr = problem(t, rng)
            for k in coef:
                coef[k].append(pr[k])
    trees.append(np.zeros(0, np.int32))  # an empty cell
    for k in coef:
        coef[k].append(np.zeros(0))
    ncomp = np.array([t.size for t in trees], np.int32)
    return ncomp, np.concatenate(trees), {k: np.concatenate(v) for k, v in coef.items()}


@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("per_lane", [1, 2])
def test_solve_f64_zoo(split, per_lane):
    """Both places for the FP64 factor (natural positions, block order) match
    the oracle and each other bit for bit, in both layouts."""
    ncomp, parent, c = zoo_batch(31)
    ref = oracle.solve_batch(ncomp, parent, c["d"], c["u"], c["b"])
    xs, xps = [], []
    for fp64_factor in (1, 2):
        plan = H.Plan(ncomp, parent, split_branches=split, pieces_per_lane=per_lane, fp64_factor=fp64_factor)
        x = dev(c["b"])
        H.solve(plan, dev(c["d"]), dev(c["u"]), x)
        assert cell_rel_err(x.cpu().numpy(), ref, plan.offsets).max() <= TOL_F64
        pk = [H.pack(plan, dev(c[k])) for k in ("d", "u", "b")]
        H.solve_packed(plan, *pk)
        xps.append(H.unpack(plan, pk[2]))
        xs.append(x)
        assert plan.status() == 0
    assert torch.equal(xs[0], xs[1]) and torch.equal(xps[0], xps[1]) and torch.equal(xs[0], xps[0])


def test_inputs_not_modified_and_repeatable():
    ncomp, parent, c = zoo_batch(32, sizes=(50, 400))
    plan = H.Plan(ncomp, parent)
    d, u = dev(c["d"]), dev(c["u"])
    x1 = dev(c["b"])
    H.solve(plan, d, u, x1)
    x2 = dev(c["b"])
    H.solve(plan, d, u, x2)
    assert torch.equal(d.cpu(), torch.as_tensor(c["d"])) and torch.equal(u.cpu(), torch.as_tensor(c["u"]))
    assert torch.equal(x1, x2)  # deterministic: fixed fold order, no atomics


def test_solve_golden_tiny_systems():
    from tests.test_oracle_pins import load_golden
    g = load_golden()
    trees = [v[0] for v in g.values()]
    ncomp = [t.size for t in trees]
    cat = lambda j: np.concatenate([[float(t) for t in v[j]] for v in g.values()])  # noqa: E731
    plan = H.Plan(ncomp, np.concatenate(trees))
    x = dev(cat(3))
    H.solve(plan, dev(cat(1)), dev(cat(2)), x)
    exact = cat(4)
    assert cell_rel_err(x.cpu().numpy(), exact, plan.offsets).max() < 1e-14


def test_solve_f64_fp64_small_workload():
    pop = I.population("fp64_small")
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = dev(pop["b"])
    H.solve(plan, dev(pop["d"]), dev(pop["u"]), x)
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], pop["d"], pop["u"], pop["b"])
    assert cell_rel_err(x.cpu().numpy(), ref, plan.offsets).max() <= TOL_F64


def _widened(pop):
    return {k: pop[k].astype(np.float32) for k in ("d", "u", "b")}


@pytest.mark.parametrize("name", ["fp64_small", "fp64_uniform"])
def test_solve_f32(name):
    pop = I.population(name, cells=np.arange(64))
    f = _widened(pop)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = dev(f["b"], torch.float32)
    H.solve(plan, dev(f["d"], torch.float32), dev(f["u"], torch.float32), x)
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f[k].astype(np.float64) for k in ("d", "u", "b")))
    assert cell_rel_err(x.cpu().numpy().astype(np.float64), ref, plan.offsets).max() <= TOL_F32


@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("per_lane", [1, 2])
def test_solve_refine_mixed_population(steps, per_lane):
    w = I.WORKLOADS["uneven_mixed"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:24], np.nonzero(cls == 1)[0][:3]])
    pop = I.population(w, cells=cells, margin=1e-1)
    f = _widened(pop)
    plan = H.Plan(pop["ncomp"], pop["parent"], pieces_per_lane=per_lane)
    relres = torch.empty(plan.n_cells, dtype=torch.float64, device="cuda")
    x = H.solve_refine(plan, *(dev(f[k], torch.float32) for k in ("d", "u", "b")), steps=steps, relres=relres)
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f[k].astype(np.float64) for k in ("d", "u", "b")))
    err = cell_rel_err(x.cpu().numpy(), ref, plan.offsets)
    if steps == 2:
        assert err.max() <= TOL_REFINE
    else:
        assert err.max() <= 1e-8
    assert relres.cpu().numpy().max() < (1e-12 if steps == 2 else 1e-8)
    assert plan.status() in (0, H.HINES_WARN_REFINE)


@pytest.mark.parametrize("per_lane", [1, 2])
def test_solve_refine_zoo_edge_cases(per_lane):
    ncomp, parent, c = zoo_batch(33)
    f = {k: c[k].astype(np.float32) for k in ("d", "u", "b")}
    plan = H.Plan(ncomp, parent, pieces_per_lane=per_lane)
    x = H.solve_refine(plan, *(dev(f[k], torch.float32) for k in ("d", "u", "b")), steps=2)
    ref = oracle.solve_batch(ncomp, parent, *(f[k].astype(np.float64) for k in ("d", "u", "b")))
    assert cell_rel_err(x.cpu().numpy(), ref, plan.offsets).max() <= TOL_REFINE


@pytest.mark.parametrize("theta", [0, 1])
@pytest.mark.parametrize("per_lane", [1, 2])
def test_cable_steps_match_oracle(theta, per_lane):
    w = I.WORKLOADS["uneven_steps"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:12], np.nonzero(cls == 1)[0][:2]])
    pop = I.population(w, cells=cells, keys=("s", "a", "u", "g", "V0"))
    plan = H.Plan(pop["ncomp"], pop["parent"], pieces_per_lane=per_lane)
    s, g, u = dev(pop["s"]), dev(pop["g"]), dev(pop["u"])
    V = dev(pop["V0"])
    K = 15
    for _ in range(K):
        H.cable_step(plan, s, g, u, V, w.dt, w.E, theta)
    ref, _ = oracle.steps_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"], K, w.dt, w.E,
                                theta)
    assert cell_rel_err(V.cpu().numpy(), ref, plan.offsets).max() <= TOL_F64


def test_grad_du_matches_oracle_solves():
    ncomp, parent, c = zoo_batch(34, sizes=(3, 64, 500))
    plan = H.Plan(ncomp, parent)
    rng = np.random.default_rng(5)
    xbar = rng.standard_normal(parent.size)
    x = oracle.solve_batch(ncomp, parent, c["d"], c["u"], c["b"])
    lam = oracle.solve_batch(ncomp, parent, c["d"], c["u"], xbar)
    gd, gu = H.grad_du(plan, dev(lam), dev(x))
    off = plan.offsets
    ref_d = -lam * x
    ref_u = np.zeros_like(x)
    for cc in range(len(ncomp)):
        for i in range(off[cc] + 1, off[cc + 1]):
            pi = off[cc] + parent[i]
            ref_u[i] = -(lam[i] * x[pi] + lam[pi] * x[i])
    assert np.abs(gd.cpu().numpy() - ref_d).max() <= 1e-15 * np.abs(ref_d).max()
    assert np.abs(gu.cpu().numpy() - ref_u).max() <= 1e-15 * np.abs(ref_u).max()


def test_empty_batch():
    plan = H.Plan([], np.zeros(0, np.int32))
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    H.solve(plan, e, e, e)
    torch.cuda.synchronize()


def test_wrong_device_arguments_rejected():
    plan = H.Plan([3], np.array([-1, 0, 1], np.int32))
    with pytest.raises(TypeError):
        H.solve(plan, torch.zeros(3, dtype=torch.float64), torch.zeros(3, dtype=torch.float64),
                torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError):
        H.solve(plan, dev(np.zeros(4)), dev(np.zeros(4)), dev(np.zeros(4)))


@pytest.mark.parametrize("per_lane", [1, 2])
def test_solve_compensated_zoo_edge_cases(per_lane):
    ncomp, parent, c = zoo_batch(35)
    f = {k: c[k].astype(np.float32) for k in ("d", "u", "b")}
    for split in (0, 1, 2):
        plan = H.Plan(ncomp, parent, split_branches=split, pieces_per_lane=per_lane)
        x = H.solve_compensated(plan, *(dev(f[k], torch.float32) for k in ("d", "u", "b")))
        ref = oracle.solve_batch(ncomp, parent, *(f[k].astype(np.float64) for k in ("d", "u", "b")))
        assert cell_rel_err(x.cpu().numpy(), ref, plan.offsets).max() <= TOL_REFINE


@pytest.mark.parametrize("margin", [
    1e-1,
    1e-3,
    pytest.param(1e-5, marks=pytest.mark.xfail(
        strict=True, reason="at margin 1e-5 (Skeel condition ~9e5) the compensated solve reaches about 3.3e-10 "
                            "against the oracle: above the 1e-10 gate; the refined path must be used there")),
])
def test_solve_compensated_margin_sweep(margin):
    """Leak margins of the mixed-precision workload, every cell held to the
    FP32-input gate 1e-10.  Double-float arithmetic carries about 48 bits, so
    the error grows like cond * 2^-48; at margin 1e-5 the compensated solve
    misses the gate (an expected, strict failure)."""
    w = I.WORKLOADS["uneven_mixed"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:24], np.nonzero(cls == 1)[0][:3]])
    pop = I.population(w, cells=cells, margin=margin)
    f = _widened(pop)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = H.solve_compensated(plan, *(dev(f[k], torch.float32) for k in ("d", "u", "b")))
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f[k].astype(np.float64) for k in ("d", "u", "b")))
    assert cell_rel_err(x.cpu().numpy(), ref, plan.offsets).max() <= TOL_REFINE


@pytest.mark.parametrize("margin,steps", [(1e-1, 1), (1e-1, 2), (1e-3, 2), (1e-5, 4)])
def test_solve_refine_margin_sweep(margin, steps):
    """FP32 elimination with refinement steps against the oracle at the
    leak margins where the refinement reaches the 1e-10 gate (one step at
    margin 0.1, two at 1e-3, four at 1e-5, on the same 256 cells the bench's
    sweep uses)."""
    w = I.WORKLOADS["uneven_mixed"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:180], np.nonzero(cls == 1)[0][:76]])
    pop = I.population(w, cells=cells, margin=margin)
    f = _widened(pop)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = H.solve_refine(plan, *(dev(f[k], torch.float32) for k in ("d", "u", "b")), steps=steps)
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f[k].astype(np.float64) for k in ("d", "u", "b")))
    assert cell_rel_err(x.cpu().numpy(), ref, plan.offsets).max() <= TOL_REFINE


def test_solve_compensated_deterministic():
    ncomp, parent, c = zoo_batch(36, sizes=(200, 1500))
    f = {k: dev(c[k].astype(np.float32), torch.float32) for k in ("d", "u", "b")}
    plan = H.Plan(ncomp, parent)
    x1 = H.solve_compensated(plan, f["d"], f["u"], f["b"])
    x2 = H.solve_compensated(plan, f["d"], f["u"], f["b"])
    assert torch.equal(x1, x2)
