"""The pins must catch plausible mistakes: each case plants one mistake in a
private copy of the oracle source (on the CPU), rebuilds it and checks that an
independent pin rejects the mutant while the unmutated build passes."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

from paper_1810_12742_gb300 import inputs as I
from tests.helpers import dense, problem, tree_zoo

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "hines_oracle.c")

MUTATIONS = {
    "none": None,
    "listing2_literal_u_of_parent": ("d[par] -= l * u[row];", "d[par] -= l * u[par];"),
    "rhs_sign": ("b[par] -= l * b[row];", "b[par] += l * b[row];"),
    "forward_dropped_term": ("const double known = row == 0 ? 0.0 : u[row] * b[p[row]];", "const double known = 0.0;"),
    "forward_thomas_index": ("u[row] * b[p[row]];", "u[row] * b[row - 1];"),
    "matvec_missing_transpose": ("y[p[i]] = y[p[i]] + u[i] * x[i];", ""),
    "rebuild_missing_parent_edge": ("d[p[i]] = d[p[i]] + a[i];", ""),
    "adjoint_grad_a_sign": ("grad_a[lo + i] = grad_a[lo + i] - (lam[i]", "grad_a[lo + i] = grad_a[lo + i] + (lam[i]"),
    "adjoint_old_state": ("double dLdd = -lam[i] * Vk[i];", "double dLdd = -lam[i] * Vm[i];"),
    "adjoint_no_chain": ("vbar[i] = lam[i] * sc[i] * (1.0 - (1.0 - (double)theta) * dt * gc[i]);", "vbar[i] = 0.0;"),
}


def _build(tmp_path, name):
    src = open(SRC).read()
    mut = MUTATIONS[name]
    if mut is not None:
        assert mut[0] in src, name
        src = src.replace(mut[0], mut[1], 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(c),
                           "-lm"])
    L = ctypes.CDLL(str(so))
    vp = ctypes.c_void_p
    L.oracle_hines.argtypes = [ctypes.c_int64, vp, vp, vp, vp]
    L.oracle_matvec.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp]
    L.oracle_adjoint_batch.argtypes = [ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, vp, vp, vp, ctypes.c_int]
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pins_pass(L):
    rng = np.random.default_rng(5)
    ok = True
    for _, p in tree_zoo(rng, 60).items():
        pr = problem(p, rng)
        p = np.ascontiguousarray(p, np.int32)
        d, u, b = pr["d"].copy(), pr["u"].copy(), pr["b"].copy()
        L.oracle_hines(p.size, _ptr(p), _ptr(d), _ptr(u), _ptr(b))
        A = dense(p, pr["d"], pr["u"])
        ok &= np.abs(b - np.linalg.solve(A, pr["b"])).max() < 1e-12
        x = rng.standard_normal(p.size)
        y = np.empty_like(x)
        L.oracle_matvec(p.size, _ptr(p), _ptr(pr["d"]), _ptr(pr["u"]), _ptr(x), _ptr(y))
        ok &= np.abs(y - A @ x).max() < 1e-12
    # adjoint against dense torch autograd on one small cell
    p = I.random_chainy_tree(rng, 25)
    n = p.size
    a = rng.uniform(0.5, 2, n)
    s = rng.uniform(0.01, 0.1, n)
    g = rng.uniform(0.1, 1, n)
    V0 = rng.uniform(-80, -50, n)
    tgt = np.array([-60.0])
    off = np.array([0, n], np.int64)
    loss, gg, ga = np.zeros(1), np.zeros(n), np.zeros(n)
    L.oracle_adjoint_batch(1, _ptr(off), _ptr(p), _ptr(s), _ptr(g), _ptr(a), _ptr(V0), _ptr(tgt), 6, 0.025, -65.0, 1,
                           _ptr(loss), _ptr(gg), _ptr(ga), 1)
    gt = torch.tensor(g, requires_grad=True)
    at = torch.tensor(a, requires_grad=True)
    idx = torch.arange(1, n)
    pt = torch.as_tensor(p[1:].astype(np.int64))
    W = torch.zeros(n, n, dtype=torch.float64).index_put((idx, pt), at[1:]).index_put((pt, idx), at[1:], accumulate=True)
    A = torch.diag(torch.as_tensor(s) * (1 + 0.025 * gt)) + torch.diag(W.sum(1)) - W
    V = torch.as_tensor(V0)
    Lt = 0
    for _ in range(6):
        V = torch.linalg.solve(A, torch.as_tensor(s) * V + torch.as_tensor(s) * 0.025 * gt * -65.0)
        Lt = Lt + (V[0] + 60.0) ** 2
    Lt.backward()
    ok &= abs(loss[0] - Lt.item()) < 1e-9 * Lt.item()
    ok &= np.abs(gg - gt.grad.numpy()).max() < 1e-9 * np.abs(gg).max()
    ok &= np.abs(ga[1:] - at.grad.numpy()[1:]).max() < 1e-9 * np.abs(ga).max()
    return bool(ok)


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_pins_catch_mutant(tmp_path, name):
    L = _build(tmp_path, name)
    assert _pins_pass(L) == (name == "none")
