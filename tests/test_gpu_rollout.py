"""Passive-cable time stepping (CUDA graph) and the adjoint, against the
oracle's stepper and its independent adjoint."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I
from paper_1810_12742_gb300 import rollout as R
from tests.helpers import problem, tree_zoo

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rel_cells(x, ref, off):
    e = 0.0
    for c in range(len(off) - 1):
        sl = slice(off[c], off[c + 1])
        if off[c + 1] > off[c]:
            e = max(e, np.abs(x[sl] - ref[sl]).max() / np.abs(ref[sl]).max())
    return e


def uneven_subset(n_small, n_large, keys=("s", "a", "u", "g", "V0", "target")):
    w = I.WORKLOADS["uneven_steps"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:n_small], np.nonzero(cls == 1)[0][:n_large]])
    return w, I.population(w, cells=cells, keys=keys)


def test_graph_replay_equals_eager_and_oracle():
    w, pop = uneven_subset(20, 2)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    s, g, u = dev(pop["s"]), dev(pop["g"]), dev(pop["u"])
    V_eager = dev(pop["V0"])
    for _ in range(30):
        H.cable_step(plan, s, g, u, V_eager, w.dt, w.E, 1)
    V_graph = dev(pop["V0"])
    st = R.CableStepper(plan, s, g, u, V_graph, w.dt, w.E, 1, steps=10)
    for _ in range(3):
        st.replay()
    torch.cuda.synchronize()
    assert torch.equal(V_graph, V_eager)
    ref, _ = oracle.steps_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"], 30, w.dt, w.E, 1)
    assert rel_cells(V_graph.cpu().numpy(), ref, plan.offsets) <= 1e-12


def test_thousand_steps_uneven_subset():
    """The 1000-step rollout of the uneven population on a seeded subset of
    small and large cells (cells are independent)."""
    w, pop = uneven_subset(48, 4)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    s, g, u = dev(pop["s"]), dev(pop["g"]), dev(pop["u"])
    V = dev(pop["V0"])
    st = R.CableStepper(plan, s, g, u, V, w.dt, w.E, 1, steps=w.steps)
    st.replay()
    torch.cuda.synchronize()
    ref, _ = oracle.steps_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"], w.steps, w.dt,
                                w.E, 1, nthreads=8)
    assert rel_cells(V.cpu().numpy(), ref, plan.offsets) <= 1e-12


@pytest.mark.parametrize("theta", [0, 1])
@pytest.mark.parametrize("fp64_factor", [1, 2])
def test_solver_layout_steps_equal_natural(theta, fp64_factor):
    """hines_cable_step_packed / hines_cable_solve_packed give the natural-layout
    results bit for bit; the graph stepper in the solver layout too; for both
    places of the factor."""
    w, pop = uneven_subset(24, 2)
    plan = H.Plan(pop["ncomp"], pop["parent"], fp64_factor=fp64_factor)
    s, g, u = dev(pop["s"]), dev(pop["g"]), dev(pop["u"])
    V = dev(pop["V0"])
    pk = [H.pack(plan, t) for t in (s, g, u, V)]
    for _ in range(5):
        H.cable_step(plan, s, g, u, V, w.dt, w.E, theta)
        H.cable_step_packed(plan, pk[0], pk[1], pk[2], pk[3], w.dt, w.E, theta)
    assert torch.equal(H.unpack(plan, pk[3]), V)
    y = V.clone()
    yp = H.pack(plan, y)
    H.cable_solve(plan, s, g, u, y, w.dt, theta)
    H.cable_solve_packed(plan, pk[0], pk[1], pk[2], yp, w.dt, theta)
    assert torch.equal(H.unpack(plan, yp), y)
    V1, V2 = dev(pop["V0"]), dev(pop["V0"])
    a = R.CableStepper(plan, s, g, u, V1, w.dt, w.E, theta, steps=7)
    b = R.CableStepper(plan, s, g, u, V2, w.dt, w.E, theta, steps=7, layout="solver")
    a.replay()
    b.replay()
    assert torch.equal(b.fetch(), V1)


@pytest.mark.parametrize("theta", [0, 1])
def test_cable_steps_reusing_the_factor_equal_full_steps(theta):
    """After one full step the passive cable's factor serves later steps
    (the matrix is constant): bit-identical states, both layouts, eager and
    in the graph stepper."""
    w, pop = uneven_subset(24, 2)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    s, g, u = dev(pop["s"]), dev(pop["g"]), dev(pop["u"])
    Vf, Vr = dev(pop["V0"]), dev(pop["V0"])
    for k in range(6):
        H.cable_step(plan, s, g, u, Vf, w.dt, w.E, theta)
    H.cable_step(plan, s, g, u, Vr, w.dt, w.E, theta)
    for k in range(5):
        H.cable_step_reuse(plan, s, g, u, Vr, w.dt, w.E, theta)
    assert torch.equal(Vf, Vr)
    pk = [H.pack(plan, t) for t in (s, g, u)]
    Vp = H.pack(plan, dev(pop["V0"]))
    H.cable_step_packed(plan, *pk, Vp, w.dt, w.E, theta)
    for k in range(5):
        H.cable_step_reuse(plan, *pk, Vp, w.dt, w.E, theta, solver_layout=True)
    assert torch.equal(H.unpack(plan, Vp), Vf)
    for layout in ("natural", "solver"):
        V1, V2 = dev(pop["V0"]), dev(pop["V0"])
        a = R.CableStepper(plan, s, g, u, V1, w.dt, w.E, theta, steps=6, layout=layout)
        b = R.CableStepper(plan, s, g, u, V2, w.dt, w.E, theta, steps=6, layout=layout, reuse_factor=True)
        a.replay()
        b.replay()
        assert torch.equal(a.fetch(), b.fetch())


@pytest.mark.parametrize("theta", [0, 1])
@pytest.mark.parametrize("layout", ["natural", "solver"])
@pytest.mark.parametrize("fp64_factor", [1, 2])
def test_cable_steps_reusing_the_factor_match_oracle(theta, layout, fp64_factor):
    """The factor-reuse variant against the oracle's own stepper directly (not
    only against the full steps): one full step, then steps that eliminate
    only the rebuilt right-hand side with the stored factor, wherever the plan
    keeps it (natural positions or block order)."""
    w, pop = uneven_subset(20, 2)
    plan = H.Plan(pop["ncomp"], pop["parent"], fp64_factor=fp64_factor)
    s, g, u = dev(pop["s"]), dev(pop["g"]), dev(pop["u"])
    K = 12
    if layout == "natural":
        V = dev(pop["V0"])
        H.cable_step(plan, s, g, u, V, w.dt, w.E, theta)
        for _ in range(K - 1):
            H.cable_step_reuse(plan, s, g, u, V, w.dt, w.E, theta)
    else:
        pk = [H.pack(plan, s), H.pack(plan, g), H.pack_coupling(plan, u)]
        Vp = H.pack(plan, dev(pop["V0"]))
        H.cable_step_packed(plan, *pk, Vp, w.dt, w.E, theta)
        for _ in range(K - 1):
            H.cable_step_reuse(plan, *pk, Vp, w.dt, w.E, theta, solver_layout=True)
        V = H.unpack(plan, Vp)
    ref, _ = oracle.steps_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"], K, w.dt, w.E,
                                theta)
    assert rel_cells(V.cpu().numpy(), ref, plan.offsets) <= 1e-12


def _adjoint_case(cells, steps, ce, theta=1):
    w = I.WORKLOADS["adjoint"]
    pop = I.population(w, cells=cells, keys=("s", "a", "u", "g", "V0", "target"))
    plan = H.Plan(pop["ncomp"], pop["parent"])
    t = {k: dev(pop[k]) for k in ("s", "a", "g", "V0", "target")}
    ga = t["g"].clone().requires_grad_(True)
    aa = t["a"].clone().requires_grad_(True)
    L = R.CableRollout.apply(ga, aa, plan, t["s"], t["V0"], t["target"], steps, w.dt, w.E, theta, ce)
    L.backward()
    loss, rg, ra = oracle.adjoint_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"],
                                        pop["target"], steps, w.dt, w.E, theta, nthreads=8)
    return plan, pop, L.item(), ga.grad.cpu().numpy(), aa.grad.cpu().numpy(), loss, rg, ra


@pytest.mark.parametrize("theta", [0, 1])
def test_adjoint_matches_oracle_small(theta):
    plan, pop, L, gg, ga, loss, rg, ra = _adjoint_case(np.arange(6), 40, 10, theta)
    assert abs(L - loss.sum()) <= 1e-11 * loss.sum()
    mask = np.ones(ga.size, bool)
    mask[plan.offsets[:-1]] = False
    assert np.abs(gg - rg).max() <= 1e-10 * np.abs(rg).max()
    assert np.abs(ga[mask] - ra[mask]).max() <= 1e-10 * np.abs(ra).max()


def test_adjoint_full_workload_matches_oracle_gradient():
    """256 cells x U[100,500] branches x 16 compartments, 200 steps, checkpoints
    every 20 steps: loss and both gradients against the oracle's adjoint."""
    w = I.WORKLOADS["adjoint"]
    plan, pop, L, gg, ga, loss, rg, ra = _adjoint_case(np.arange(w.n_cells), w.steps, w.checkpoint_every)
    assert abs(L - loss.sum()) <= 1e-11 * loss.sum()
    mask = np.ones(ga.size, bool)
    mask[plan.offsets[:-1]] = False
    for c in range(plan.n_cells):  # per cell, relative to that cell's largest gradient
        sl = slice(plan.offsets[c], plan.offsets[c + 1])
        assert np.abs(gg[sl] - rg[sl]).max() <= 1e-10 * np.abs(rg[sl]).max()
        m = mask[sl]
        assert np.abs(ga[sl][m] - ra[sl][m]).max() <= 1e-10 * np.abs(ra[sl][m]).max()


def test_adjoint_central_differences_on_gpu_forward():
    w = I.WORKLOADS["adjoint"]
    cells = np.arange(3)
    pop = I.population(w, cells=cells, keys=("s", "a", "u", "g", "V0", "target"))
    plan = H.Plan(pop["ncomp"], pop["parent"])
    t = {k: dev(pop[k]) for k in ("s", "a", "g", "V0", "target")}
    K, ce = 40, 10

    def loss(gv, av):
        lc, _, _ = R.cable_rollout(plan, t["s"], gv, -av, t["V0"], t["target"], K, w.dt, w.E, 1, ce)
        return lc.sum().item()

    ga = t["g"].clone().requires_grad_(True)
    aa = t["a"].clone().requires_grad_(True)
    L = R.CableRollout.apply(ga, aa, plan, t["s"], t["V0"], t["target"], K, w.dt, w.E, 1, ce)
    L.backward()
    rng = np.random.default_rng(3)
    h = 1e-6
    eps_L = 2048 * 2.0 ** -52 * L.item() / h  # rounding of L itself dominates at h = 1e-6
    for i in rng.choice(plan.n_unknowns, 6, replace=False):
        e = torch.zeros_like(t["g"])
        e[i] = h
        fd = (loss(t["g"] + e, t["a"]) - loss(t["g"] - e, t["a"])) / (2 * h)
        assert abs(fd - ga.grad[i].item()) <= 1e-5 * abs(ga.grad[i].item()) + eps_L
    for i in rng.choice(np.setdiff1d(np.arange(plan.n_unknowns), plan.offsets[:-1]), 6, replace=False):
        e = torch.zeros_like(t["a"])
        e[i] = h
        fd = (loss(t["g"], t["a"] + e) - loss(t["g"], t["a"] - e)) / (2 * h)
        assert abs(fd - aa.grad[i].item()) <= 1e-5 * abs(aa.grad[i].item()) + eps_L


def test_rollout_graphs_equal_eager_rollout():
    """The captured forward and reverse graphs give the eager rollout's loss
    and gradients bit for bit, and a second replay with new inputs follows
    the new inputs (the graphs read their static buffers, not stale data)."""
    w = I.WORKLOADS["adjoint"]
    pop = I.population(w, cells=np.arange(5), keys=("s", "a", "u", "g", "V0", "target"))
    plan = H.Plan(pop["ncomp"], pop["parent"])
    t = {k: dev(pop[k]) for k in ("s", "a", "g", "V0", "target")}
    K, ce = 30, 7
    for scale in (1.0, 1.1):
        g = t["g"] * scale
        u = -t["a"]
        lc, ck, VL = R.cable_rollout(plan, t["s"], g, u, t["V0"], t["target"], K, w.dt, w.E, 1, ce)
        gg, ga = R.cable_rollout_grad(plan, t["s"], g, u, t["target"], K, w.dt, w.E, 1, ce, ck, VL)
        rg = R.rollout_graphs(plan, K, w.dt, w.E, 1, ce)
        loss = rg.forward(g, u, t["s"], t["V0"], t["target"])
        assert torch.equal(loss, lc)
        g2, a2 = rg.backward()
        assert torch.equal(g2, gg) and torch.equal(a2, ga)


def test_hines_solve_autograd_gradcheck():
    rng = np.random.default_rng(4)
    trees = list(tree_zoo(rng, 9).values())
    ncomp = [t.size for t in trees]
    parent = np.concatenate(trees)
    prs = [problem(t, rng) for t in trees]
    cat = lambda k: np.concatenate([p[k] for p in prs])  # noqa: E731
    plan = H.Plan(ncomp, parent)
    d = dev(cat("d")).requires_grad_(True)
    u = dev(cat("u")).requires_grad_(True)
    b = dev(cat("b")).requires_grad_(True)
    mask = torch.ones(parent.size, dtype=torch.float64, device="cuda")
    mask[torch.as_tensor(plan.offsets[:-1])] = 0.0  # u at a cell root is not part of A

    def f(d, u, b):
        return R.HinesSolve.apply(plan, d, u * mask + u.detach() * (1 - mask), b)

    assert torch.autograd.gradcheck(f, (d, u, b), eps=1e-6, atol=1e-8, rtol=1e-6)
