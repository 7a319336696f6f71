"""Time stepping, CUDA-graph capture and adjoints on top of the C-ABI.

Every numerical step runs in libhines kernels; this module only orders the
calls, captures them in a CUDA graph and keeps the checkpoints.

* ``CableStepper``: K fused rebuild + solve steps of the passive cable
  (hines_cable_step) captured once in a CUDA graph and replayed.
* ``cable_rollout`` / ``cable_rollout_grad``: loss
  L = sum over cells and steps of (V_root^k - target)^2 and its gradient with
  respect to the leak conductance g and the axial coefficients a (u = -a),
  with the states checkpointed every ``checkpoint_every`` steps and each
  segment recomputed during the reverse sweep.  The matrix is symmetric, so
  the adjoint of a step is one more Hines solve (hines_cable_solve).
* ``RolloutGraphs``: the same forward rollout and reverse sweep, each
  captured once in a CUDA graph over static buffers and replayed (a rollout
  of a small batch is hundreds of short launches; the graph removes their
  launch cost).
* ``HinesSolve`` and ``CableRollout``: torch.autograd.Function wrappers
  (``CableRollout`` replays the graphs of ``RolloutGraphs``).
"""
from __future__ import annotations

import weakref

import torch

from . import hines as H


class CableStepper:
    """``steps`` implicit-Euler steps of the passive cable, captured in one CUDA
    graph; ``replay()`` advances the state by ``steps`` steps.

    layout "natural": the graph steps the caller's V in place.  layout
    "solver": s, g, u and V are permuted once into the solver layout
    (Section 5) and the graph steps that copy; ``fetch()`` writes the state
    back into the caller's V.  reuse_factor: every replay makes one full step
    and then steps that re-use its factor (hines_cable_step_reuse; the
    passive cable's matrix does not change), with the same results."""

    def __init__(self, plan: H.Plan, s, g, u, V, dt: float, E: float, theta: int = 1, steps: int = 1000,
                 layout: str = "natural", reuse_factor: bool = False):
        if layout not in ("natural", "solver"):
            raise ValueError(f"layout: expected 'natural' or 'solver', got {layout!r}")
        self.plan, self.V, self.layout = plan, V, layout
        self.steps = steps
        packed = layout == "solver"
        if packed:
            self.pk = [H.pack(plan, s), H.pack(plan, g), H.pack_coupling(plan, u), H.pack(plan, V)]
            s, g, u, state = self.pk
        else:
            state = V

        def full(Vt):
            (H.cable_step_packed if packed else H.cable_step)(plan, s, g, u, Vt, dt, E, theta)

        def reuse(Vt):  # the matrix is constant: the factor of the replay's first step serves the rest
            H.cable_step_reuse(plan, s, g, u, Vt, dt, E, theta, solver_layout=packed)
        # one eager step on a scratch copy creates the kernels' resources before capture
        full(state.clone())
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            for k in range(steps):
                (reuse if reuse_factor and k > 0 else full)(state)

    def replay(self):
        self.graph.replay()

    def fetch(self):
        """The current state in the caller's V (natural layout)."""
        if self.layout == "solver":
            H.unpack(self.plan, self.pk[3], self.V)
        return self.V


def cable_rollout(plan: H.Plan, s, g, u, V0, target, steps: int, dt: float, E: float, theta: int = 1,
                  checkpoint_every: int = 20):
    """Forward rollout.  Returns (loss per cell, checkpoints) where
    checkpoints[j] is V at step j * checkpoint_every."""
    V = V0.clone()
    loss = torch.zeros(plan.n_cells, dtype=torch.float64, device=V.device)
    ckpt = [V0.clone()]
    for k in range(1, steps + 1):
        H.cable_step(plan, s, g, u, V, dt, E, theta)
        H.lib().hines_cable_loss_accumulate(plan.handle, H._dptr(V, torch.float64, plan.n_unknowns, "V"),
                                            H._dptr(target, torch.float64, plan.n_cells, "target"),
                                            H._dptr(loss, torch.float64, plan.n_cells, "loss"), H._stream())
        if k % checkpoint_every == 0 and k < steps:
            ckpt.append(V.clone())
    return loss, ckpt, V


def cable_rollout_grad(plan: H.Plan, s, g, u, target, steps: int, dt: float, E: float, theta: int,
                       checkpoint_every: int, ckpt, V_last):
    """Reverse sweep with segment recomputation.  Returns (dL/dg, dL/da)."""
    n = plan.n_unknowns
    dev = s.device
    grad_g = torch.zeros(n, dtype=torch.float64, device=dev)
    grad_a = torch.zeros(n, dtype=torch.float64, device=dev)
    vbar = torch.zeros(n, dtype=torch.float64, device=dev)
    H.cable_loss_seed(plan, V_last, target, vbar)
    lam = torch.empty_like(vbar)
    nseg = (steps + checkpoint_every - 1) // checkpoint_every
    for seg in range(nseg - 1, -1, -1):
        k0 = seg * checkpoint_every
        k1 = min(steps, k0 + checkpoint_every)
        states = [ckpt[seg].clone()]
        for _ in range(k0, k1):
            V = states[-1].clone()
            H.cable_step(plan, s, g, u, V, dt, E, theta)
            states.append(V)
        for k in range(k1, k0, -1):
            lam.copy_(vbar)
            H.cable_solve(plan, s, g, u, lam, dt, theta)
            H.cable_adjoint_step(plan, lam, states[k - k0], states[k - 1 - k0], s, g, target, dt, E, theta,
                                 int(k - 1 >= 1), grad_g, grad_a, vbar)
    return grad_g, grad_a


class RolloutGraphs:
    """The forward rollout and the checkpointed reverse sweep of
    ``cable_rollout`` / ``cable_rollout_grad``, each captured once in a CUDA
    graph over static buffers.  ``forward(g, u, s, V0, target)`` copies the
    inputs in and replays the forward graph (loss per cell, checkpoints and
    the last state stay in the object's buffers); ``backward()`` replays the
    reverse sweep on them and returns (dL/dg, dL/da) buffers.  The same
    kernels run in the same order as the eager functions, so the results are
    bit-identical to them."""

    def __init__(self, plan: H.Plan, steps: int, dt: float, E: float, theta: int, checkpoint_every: int):
        # the plan owns this object (rollout_graphs keeps it on the plan), so
        # only a weak reference goes back: no reference cycle keeps a plan
        # alive until the cycle collector frees it at an arbitrary moment
        self._plan = weakref.ref(plan)
        self.cfg = (steps, dt, E, theta, checkpoint_every)
        n, nc = plan.n_unknowns, plan.n_cells
        f = dict(dtype=torch.float64, device="cuda")
        self.g, self.u, self.s, self.V0 = (torch.zeros(n, **f) for _ in range(4))
        self.target = torch.zeros(nc, **f)
        self.loss = torch.zeros(nc, **f)
        nseg = (steps + checkpoint_every - 1) // checkpoint_every
        self.ckpt = [torch.zeros(n, **f) for _ in range(nseg)]
        self.V = torch.zeros(n, **f)
        self.states = [torch.zeros(n, **f) for _ in range(checkpoint_every + 1)]
        self.grad_g, self.grad_a, self.vbar, self.lam = (torch.zeros(n, **f) for _ in range(4))
        # the first step creates nothing lazily, but run each body once eagerly
        # so that every kernel has been loaded before capture
        self._fwd_body()
        self._bwd_body()
        torch.cuda.synchronize()
        self.fwd_graph, self.bwd_graph = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.fwd_graph):
            self._fwd_body()
        with torch.cuda.graph(self.bwd_graph):
            self._bwd_body()

    @property
    def plan(self):
        return self._plan()

    def _fwd_body(self):
        plan = self.plan
        steps, dt, E, theta, ce = self.cfg
        n = plan.n_unknowns
        self.loss.zero_()
        self.V.copy_(self.V0)
        self.ckpt[0].copy_(self.V0)
        for k in range(1, steps + 1):
            H.cable_step(plan, self.s, self.g, self.u, self.V, dt, E, theta)
            H.lib().hines_cable_loss_accumulate(plan.handle, H._dptr(self.V, torch.float64, n, "V"),
                                                H._dptr(self.target, torch.float64, plan.n_cells, "target"),
                                                H._dptr(self.loss, torch.float64, plan.n_cells, "loss"), H._stream())
            if k % ce == 0 and k < steps:
                self.ckpt[k // ce].copy_(self.V)

    def _bwd_body(self):
        plan = self.plan
        steps, dt, E, theta, ce = self.cfg
        s, g, u, target = self.s, self.g, self.u, self.target
        self.grad_g.zero_()
        self.grad_a.zero_()
        self.vbar.zero_()
        H.cable_loss_seed(plan, self.V, target, self.vbar)
        for seg in range(len(self.ckpt) - 1, -1, -1):
            k0 = seg * ce
            k1 = min(steps, k0 + ce)
            self.states[0].copy_(self.ckpt[seg])
            for j in range(k1 - k0):
                self.states[j + 1].copy_(self.states[j])
                H.cable_step(plan, s, g, u, self.states[j + 1], dt, E, theta)
            for k in range(k1, k0, -1):
                self.lam.copy_(self.vbar)
                H.cable_solve(plan, s, g, u, self.lam, dt, theta)
                H.cable_adjoint_step(plan, self.lam, self.states[k - k0], self.states[k - 1 - k0], s, g, target, dt,
                                     E, theta, int(k - 1 >= 1), self.grad_g, self.grad_a, self.vbar)

    def forward(self, g, u, s, V0, target):
        for dst, src in ((self.g, g), (self.u, u), (self.s, s), (self.V0, V0), (self.target, target)):
            dst.copy_(src)
        self.fwd_graph.replay()
        return self.loss

    def backward(self):
        self.bwd_graph.replay()
        return self.grad_g, self.grad_a


def rollout_graphs(plan: H.Plan, steps: int, dt: float, E: float, theta: int, checkpoint_every: int):
    """The plan's RolloutGraphs for this configuration (built on first use,
    then kept on the plan object)."""
    cache = plan.__dict__.setdefault("_rollout_graphs", {})
    key = (int(steps), float(dt), float(E), int(theta), int(checkpoint_every))
    if key not in cache:
        cache[key] = RolloutGraphs(plan, *key)
    return cache[key]


class CableRollout(torch.autograd.Function):
    """loss = CableRollout.apply(g, a, plan, s, V0, target, steps, dt, E, theta, checkpoint_every)

    Forward and backward replay the plan's captured rollout graphs
    (``rollout_graphs``); the returned gradients are copies of the graphs'
    buffers.  Two rollouts on the same plan and configuration share those
    buffers, so one's backward must run before the other's forward."""

    @staticmethod
    def forward(ctx, g, a, plan, s, V0, target, steps, dt, E, theta=1, checkpoint_every=20):
        rg = rollout_graphs(plan, steps, dt, E, theta, checkpoint_every)
        loss = rg.forward(g.detach(), torch.neg(a.detach()), s, V0, target)
        ctx.rg = rg
        return loss.sum()

    @staticmethod
    def backward(ctx, gL):
        grad_g, grad_a = ctx.rg.backward()
        return gL * grad_g, gL * grad_a, None, None, None, None, None, None, None, None, None


class HinesSolve(torch.autograd.Function):
    """x = HinesSolve.apply(plan, d, u, b): FP64 solve with its adjoint.
    Backward: lambda = A^{-1} xbar (a second solve, A symmetric); db = lambda,
    dd = -lambda x, du_i = -(lambda_i x_p(i) + lambda_p(i) x_i)."""

    @staticmethod
    def forward(ctx, plan, d, u, b):
        x = b.detach().clone()
        H.solve(plan, d.detach(), u.detach(), x)
        ctx.plan = plan
        ctx.save_for_backward(d, u, x)
        return x

    @staticmethod
    def backward(ctx, xbar):
        d, u, x = ctx.saved_tensors
        lam = xbar.detach().contiguous().clone()
        H.solve(ctx.plan, d.detach(), u.detach(), lam)
        gd, gu = H.grad_du(ctx.plan, lam, x)
        return None, gd, gu, lam
