"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to mathematics or to an independent routine:
LAPACK dense solves, exact rational arithmetic, the banded LAPACK solver,
closed-form solutions, invariants of symmetric M-matrices, and a dense
PyTorch autograd computation for the adjoint.
"""
import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
from oracle import exact
from paper_1810_12742_gb300 import inputs as I
from tests.helpers import dense, problem, relabel, tree_zoo


def rel(x, y):
    return np.abs(np.asarray(x) - np.asarray(y)).max() / max(np.abs(np.asarray(y)).max(), 1e-300)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 40, 200])
def test_matches_lapack_dense(n):
    """Section 2: the Hines algorithm solves A x = b exactly up to rounding."""
    rng = np.random.default_rng(100 + n)
    for name, p in tree_zoo(rng, n).items():
        pr = problem(p, rng)
        x = oracle.hines(p, pr["d"], pr["u"], pr["b"])
        xr = np.linalg.solve(dense(p, pr["d"], pr["u"]), pr["b"])
        assert rel(x, xr) < 1e-13, name


def test_matches_lapack_dense_mixed_signs():
    """The algorithm does not rely on the sign of the couplings."""
    rng = np.random.default_rng(7)
    for name, p in tree_zoo(rng, 120).items():
        pr = problem(p, rng)
        u = pr["u"] * rng.choice([-1.0, 1.0], size=len(p))
        x = oracle.hines(p, pr["d"], u, pr["b"])
        xr = np.linalg.solve(dense(p, pr["d"], u), pr["b"])
        assert rel(x, xr) < 1e-13, name


@pytest.mark.parametrize("seed", range(6))
def test_matches_exact_rational(seed):
    """Exact Fraction Gaussian elimination on tiny trees (no rounding at all)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 16))
    p = I.random_recursive_tree(rng, n)
    pr = problem(p, rng)
    x = oracle.hines(p, pr["d"], pr["u"], pr["b"])
    xe = np.array([float(v) for v in exact.solve(p, pr["d"], pr["u"], pr["b"])])
    assert rel(x, xe) < 1e-14


def test_thomas_equals_hines_on_chain_and_lapack_banded():
    """Section 2: with p[i] = i-1 the Hines algorithm is the Thomas algorithm;
    Thomas itself is pinned to LAPACK's banded solver."""
    rng = np.random.default_rng(3)
    n = 500
    p = np.arange(-1, n - 1, dtype=np.int32)
    pr = problem(p, rng)
    xh = oracle.hines(p, pr["d"], pr["u"], pr["b"])
    xt = oracle.thomas(pr["d"], pr["u"], pr["b"])
    assert np.array_equal(xh, xt)  # same operations in the same order
    ab = np.zeros((3, n))
    ab[0, 1:] = pr["u"][1:]  # superdiagonal A[i-1, i] = u[i]
    ab[1] = pr["d"]
    ab[2, :-1] = pr["u"][1:]  # subdiagonal A[i, i-1] = u[i]
    xb = scipy.linalg.solve_banded((1, 1), ab, pr["b"])
    assert rel(xt, xb) < 1e-13


@pytest.mark.parametrize("n,k", [(16, 1), (64, 5), (1000, 37)])
def test_closed_form_uniform_cable(n, k):
    """Constant-coefficient sealed cable: v_i = cos(pi k (i + 1/2) / n) is an
    eigenvector with eigenvalue s + 2a(1 - cos(pi k / n)), so b = lambda v gives x = v."""
    a, s = 1.3, 0.04
    p = np.arange(-1, n - 1, dtype=np.int32)
    deg = np.full(n, 2.0)
    deg[0] = deg[-1] = 1.0
    d = s + a * deg
    u = np.full(n, -a)
    v = np.cos(np.pi * k * (np.arange(n) + 0.5) / n)
    lam = s + 2 * a * (1 - np.cos(np.pi * k / n))
    x = oracle.hines(p, d, u, lam * v)
    assert np.abs(x - v).max() < 1e-12


def test_closed_form_point_source_infinite_cable_limit():
    """A unit source in the middle of a long uniform cable decays like r^|i-j|,
    r the small root of a r^2 - (s + 2a) r + a = 0."""
    n, a, s = 4001, 1.0, 0.05
    j = n // 2
    p = np.arange(-1, n - 1, dtype=np.int32)
    deg = np.full(n, 2.0)
    deg[0] = deg[-1] = 1.0
    b = np.zeros(n)
    b[j] = 1.0
    x = oracle.hines(p, s + a * deg, np.full(n, -a), b)
    c = s + 2 * a
    r = (c - np.sqrt(c * c - 4 * a * a)) / (2 * a)
    alpha = 1.0 / (c - 2 * a * r)
    idx = np.arange(j - 200, j + 201)
    assert rel(x[idx], alpha * r ** np.abs(idx - j)) < 1e-12


def test_constant_vector_any_tree():
    """With d = s + sum of a and u = -a, A 1 = s on every tree: b = k s gives x = k."""
    rng = np.random.default_rng(11)
    for name, p in tree_zoo(rng, 3000).items():
        pr = problem(p, rng)
        x = oracle.hines(p, pr["d"], pr["u"], -65.0 * pr["s"])
        assert np.abs(x + 65.0).max() < 1e-10, name


def test_invariants():
    rng = np.random.default_rng(12)
    for name, p in tree_zoo(rng, 150).items():
        n = len(p)
        pr = problem(p, rng)
        A = dense(p, pr["d"], pr["u"])
        x = oracle.hines(p, pr["d"], pr["u"], pr["b"])
        # scaled residual
        r = pr["b"] - A @ x
        assert np.abs(r).max() / (np.abs(A).sum(1).max() * np.abs(x).max()) < 10 * n * 2.0 ** -53, name
        # symmetry of the inverse
        i, j = 3 % n, (n * 2) // 3
        ei, ej = np.eye(n)[i], np.eye(n)[j]
        assert abs(oracle.hines(p, pr["d"], pr["u"], ej)[i] - oracle.hines(p, pr["d"], pr["u"], ei)[j]) < 1e-14
        # sign flip: a tree is bipartite, S A(+a) S = A(-a) with S = diag(+-1 by depth parity)
        depth = np.zeros(n, int)
        for k in range(1, n):
            depth[k] = depth[p[k]] + 1
        S = np.where(depth % 2 == 0, 1.0, -1.0)
        xf = oracle.hines(p, pr["d"], -pr["u"], S * pr["b"])
        assert rel(xf, S * x) < 1e-13, name
        # M-matrix: b >= 0 gives x >= 0; discrete maximum principle
        bp = np.abs(pr["b"])
        assert (oracle.hines(p, pr["d"], pr["u"], bp) >= 0).all()
        q = pr["b"] / pr["s"]
        xq = oracle.hines(p, pr["d"], pr["u"], pr["b"])
        assert q.min() - 1e-9 <= xq.min() and xq.max() <= q.max() + 1e-9


def test_relabelled_tree_permutes_solution():
    """Another Hines numbering of the same tree gives the same solution, permuted."""
    rng = np.random.default_rng(13)
    for name, p in tree_zoo(rng, 400).items():
        pr = problem(p, rng)
        x = oracle.hines(p, pr["d"], pr["u"], pr["b"])
        newp, perm = relabel(p, rng)
        assert oracle.check_parent(newp) == 0
        y = oracle.hines(newp, pr["d"][perm], _relabel_u(p, pr["u"], perm, newp), pr["b"][perm])
        assert rel(y, x[perm]) < 1e-12, name


def _relabel_u(p, u, perm, newp):
    # the coupling of new compartment k to its new parent is the old edge of
    # old compartment perm[k] to its old parent (DFS keeps parent edges)
    return u[perm]


def test_bad_parent_arrays_rejected():
    assert oracle.check_parent(np.array([0], np.int32)) == oracle.NOT_HINES
    assert oracle.check_parent(np.array([-1, 1], np.int32)) == oracle.NOT_HINES
    assert oracle.check_parent(np.array([-1, 0, 3, 1], np.int32)) == oracle.NOT_HINES
    assert oracle.check_parent(np.array([-1, -1], np.int32)) == oracle.NOT_HINES
    assert oracle.check_parent(np.array([-1, 0, 0, 2], np.int32)) == 0


def test_batch_equals_per_cell_and_threads():
    rng = np.random.default_rng(14)
    trees = [I.random_chainy_tree(rng, int(m)) for m in rng.integers(1, 300, 20)]
    ncomp = np.array([t.size for t in trees])
    parent = np.concatenate(trees)
    n = parent.size
    d, u, b = rng.uniform(5, 6, n), rng.uniform(-1, 0, n), rng.uniform(-1, 1, n)
    x1 = oracle.solve_batch(ncomp, parent, d, u, b, nthreads=1)
    x4 = oracle.solve_batch(ncomp, parent, d, u, b, nthreads=4)
    assert np.array_equal(x1, x4)
    off = np.concatenate(([0], np.cumsum(ncomp)))
    for c in range(len(trees)):
        sl = slice(off[c], off[c + 1])
        assert np.array_equal(x1[sl], oracle.hines(trees[c], d[sl], u[sl], b[sl]))
    y = oracle.matvec_batch(ncomp, parent, d, u, x1)
    assert np.abs(y - b).max() < 1e-13


def test_skeel_condition_matches_dense():
    rng = np.random.default_rng(15)
    p = I.random_chainy_tree(rng, 80)
    pr = problem(p, rng, (1e-3, 1e-2))
    A = dense(p, pr["d"], pr["u"])
    x = np.linalg.solve(A, pr["b"])
    ref = np.abs(np.linalg.inv(A)) @ (np.abs(A) @ np.abs(x))
    cond = oracle.skeel_batch([80], p, pr["d"], pr["u"], x)
    assert abs(cond[0] - ref.max() / np.abs(x).max()) < 1e-10 * cond[0]


# ----------------------------------------------------------------------------
# time stepping and adjoint
# ----------------------------------------------------------------------------
def _step_problem(rng, n_cells=3, n=60):
    trees = [I.random_chainy_tree(rng, n + 7 * c) for c in range(n_cells)]
    ncomp = np.array([t.size for t in trees])
    parent = np.concatenate(trees)
    N = parent.size
    a = rng.uniform(0.5, 2.0, N)
    s = rng.uniform(0.01, 0.1, N)
    g = rng.uniform(0.1, 1.0, N)
    V0 = rng.uniform(-80, -50, N)
    tgt = rng.uniform(-70, -50, n_cells)
    return ncomp, parent, a, s, g, V0, tgt


def _dense_stepper_torch(ncomp, parent, s, g, a, V0, target, nsteps, dt, E, theta):
    """Independent dense restatement with torch (CPU, float64, autograd)."""
    off = np.concatenate(([0], np.cumsum(ncomp)))
    loss = 0
    for c in range(len(ncomp)):
        lo, hi = off[c], off[c + 1]
        n = hi - lo
        p = torch.as_tensor(parent[lo:hi].astype(np.int64))
        sc = torch.as_tensor(s[lo:hi])
        gc, ac = g[lo:hi], a[lo:hi]
        A = torch.zeros(n, n, dtype=torch.float64)
        idx = torch.arange(1, n)
        A = A.index_put((idx, p[1:]), -ac[1:]).index_put((p[1:], idx), -ac[1:], accumulate=True)
        lap = -torch.diag(A.sum(1)) + A  # weighted graph Laplacian: diag(sum a), off-diagonals -a
        A = torch.diag(sc * (1 + theta * dt * gc)) + lap
        V = torch.as_tensor(V0[lo:hi])
        for _ in range(nsteps):
            b = sc * V + sc * dt * gc * (E - (1 - theta) * V)
            V = torch.linalg.solve(A, b)
            loss = loss + (V[0] - target[c]) ** 2
    return loss


@pytest.mark.parametrize("theta", [0, 1])
def test_steps_single_compartment_closed_form(theta):
    s, g, dt, E, v0 = np.array([0.05]), np.array([0.4]), 0.025, -65.0, -80.0
    V, vs = oracle.steps_batch([1], np.array([-1], np.int32), s, g, np.zeros(1), np.array([v0]), 10, dt, E, theta)
    v = v0
    for k in range(10):
        v = (v + dt * 0.4 * E) / (1 + dt * 0.4) if theta == 1 else v - dt * 0.4 * (v - E)
        assert abs(vs[k, 0] - v) < 1e-12


def test_steps_resting_state_and_uniform_decay():
    rng = np.random.default_rng(16)
    ncomp, parent, a, s, g, V0, _ = _step_problem(rng)
    V, _ = oracle.steps_batch(ncomp, parent, s, g, a, np.full(V0.size, -65.0), 25, 0.025, -65.0, 1)
    assert np.abs(V + 65.0).max() < 1e-10
    # uniform g and uniform start: the axial terms cancel, every compartment follows the point model
    gu = np.full(V0.size, 0.3)
    V, vs = oracle.steps_batch(ncomp, parent, s, gu, a, np.full(V0.size, -80.0), 5, 0.025, -65.0, 1)
    v = -80.0
    for _ in range(5):
        v = (v + 0.025 * 0.3 * -65.0) / (1 + 0.025 * 0.3)
    assert np.abs(V - v).max() < 1e-10


@pytest.mark.parametrize("theta", [0, 1])
def test_adjoint_matches_dense_torch_autograd(theta):
    rng = np.random.default_rng(17)
    ncomp, parent, a, s, g, V0, tgt = _step_problem(rng, 2, 30)
    K, dt, E = 12, 0.025, -65.0
    loss, gg, ga = oracle.adjoint_batch(ncomp, parent, s, g, a, V0, tgt, K, dt, E, theta)
    gt = torch.tensor(g, requires_grad=True)
    at = torch.tensor(a, requires_grad=True)
    L = _dense_stepper_torch(ncomp, parent, s, gt, at, V0, tgt, K, dt, E, theta)
    L.backward()
    assert abs(loss.sum() - L.item()) < 1e-10 * abs(L.item())
    off = np.concatenate(([0], np.cumsum(ncomp)))
    mask = np.ones(a.size, bool)
    mask[off[:-1]] = False  # a at a cell's first compartment is not a parameter
    assert rel(gg, gt.grad.numpy()) < 1e-10
    assert rel(ga[mask], at.grad.numpy()[mask]) < 1e-10


def test_adjoint_central_differences():
    """Central differences of the oracle's own forward loss.  Two step sizes:
    h = 1e-3 with Richardson extrapolation (truncation O(h^4), tight bound) and
    h = 1e-6 (the workload's step), whose error is dominated by the rounding of
    L itself (the states V ~ -70 carry ~1e-13 relative error after 20 solves,
    so L is known to ~1e3 eps |L|), so its bound carries that term."""
    rng = np.random.default_rng(18)
    ncomp, parent, a, s, g, V0, tgt = _step_problem(rng, 2, 40)
    K, dt, E = 20, 0.025, -65.0
    loss, gg, ga = oracle.adjoint_batch(ncomp, parent, s, g, a, V0, tgt, K, dt, E, 1)

    def L(gv, av):
        _, vs = oracle.steps_batch(ncomp, parent, s, gv, av, V0, K, dt, E, 1)
        return ((vs - tgt[None, :]) ** 2).sum()

    Lt = loss.sum()
    assert abs(L(g, a) - Lt) < 1e-9 * Lt

    def fd(fun, h):
        return (fun(h) - fun(-h)) / (2 * h)

    off = np.concatenate(([0], np.cumsum(ncomp)))
    picks = [("g", i) for i in rng.choice(g.size, 8, replace=False)]
    picks += [("a", i) for i in rng.choice(np.setdiff1d(np.arange(a.size), off[:-1]), 8, replace=False)]
    for which, i in picks:
        def fun(h, which=which, i=i):
            e = np.zeros_like(g)
            e[i] = h
            return L(g + e, a) if which == "g" else L(g, a + e)
        ref = gg[i] if which == "g" else ga[i]
        rich = (4 * fd(fun, 5e-4) - fd(fun, 1e-3)) / 3
        assert abs(rich - ref) <= 1e-7 * abs(ref) + 2048 * 2.0 ** -52 * Lt / 5e-4, (which, i)
        h = 1e-6
        assert abs(fd(fun, h) - ref) <= 1e-5 * abs(ref) + 2048 * 2.0 ** -52 * Lt / h, (which, i)


def test_dot_product_symmetry():
    """<A^{-1} y, z> = <y, A^{-1} z> for the symmetric Hines matrix."""
    rng = np.random.default_rng(19)
    p = I.random_chainy_tree(rng, 2000)
    pr = problem(p, rng)
    y, z = rng.standard_normal(2000), rng.standard_normal(2000)
    lhs = oracle.hines(p, pr["d"], pr["u"], y) @ z
    rhs = y @ oracle.hines(p, pr["d"], pr["u"], z)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def load_golden():
    """tests/golden/tiny_systems.txt: exact rational solutions (see make_golden.py)."""
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_systems.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, *fields = [t.strip() for t in line.split("|")]
        p = np.array([int(t) for t in fields[0].split(",")], np.int32)
        d, u, b, x = ([Fraction(t) for t in f.split(",")] for f in fields[1:])
        out[name] = (p, d, u, b, x)
    return out


def test_golden_exact_solutions():
    g = load_golden()
    assert len(g) == 5
    for name, (p, d, u, b, x) in g.items():
        xo = oracle.hines(p, [float(t) for t in d], [float(t) for t in u], [float(t) for t in b])
        xe = np.array([float(t) for t in x])
        assert rel(xo, xe) < 4e-16 * len(p), name
