"""Oracle for the batched Hines solver -- test infrastructure only.

A plain serial FP64 CPU implementation (``hines_oracle.c``) of what the GPU
path computes, plus an exact rational dense solver (``exact.py``) used to pin
it.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hines_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, BAD_SIZE, NOT_HINES, NOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over cells)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            i32, i64, f64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            L.oracle_check_parent.argtypes = [i64, vp]
            L.oracle_thomas.argtypes = [i64, vp, vp, vp]
            L.oracle_thomas.restype = None
            L.oracle_hines.argtypes = [i64, vp, vp, vp, vp]
            L.oracle_matvec.argtypes = [i64, vp, vp, vp, vp, vp]
            L.oracle_matvec.restype = None
            L.oracle_solve_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_int]
            L.oracle_matvec_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp]
            L.oracle_matvec_batch.restype = None
            L.oracle_skeel_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_int]
            L.oracle_steps_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_int, f64, f64, ctypes.c_int,
                                             vp, ctypes.c_int]
            L.oracle_adjoint_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int, f64, f64,
                                               ctypes.c_int, vp, vp, vp, ctypes.c_int]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def _i32(a):
    return np.ascontiguousarray(a, np.int32)


def _off(ncomp):
    off = np.zeros(len(ncomp) + 1, np.int64)
    np.cumsum(np.asarray(ncomp, np.int64), out=off[1:])
    return off


def check_parent(p) -> int:
    p = _i32(p)
    return lib().oracle_check_parent(p.size, _p(p))


def thomas(d, u, b):
    """Listing 1 (symmetric Thomas), u[i] = A[i, i-1].  Returns x."""
    d, u, b = _f64(d).copy(), _f64(u), _f64(b).copy()
    lib().oracle_thomas(d.size, _p(d), _p(u), _p(b))
    return b


def hines(p, d, u, b, return_factor: bool = False):
    """Listing 2 (symmetric Hines) on one cell.  Returns x (and the eliminated diagonal)."""
    p = _i32(p)
    d, u, b = _f64(d).copy(), _f64(u), _f64(b).copy()
    rc = lib().oracle_hines(p.size, _p(p), _p(d), _p(u), _p(b))
    if rc != OK:
        raise ValueError(f"oracle_hines: status {rc}")
    return (b, d) if return_factor else b


def matvec(p, d, u, x):
    p = _i32(p)
    d, u, x = _f64(d), _f64(u), _f64(x)
    y = np.empty_like(x)
    lib().oracle_matvec(p.size, _p(p), _p(d), _p(u), _p(x), _p(y))
    return y


def solve_batch(ncomp, parent, d, u, b, nthreads: int = 1):
    off = _off(ncomp)
    parent, d, u, b = _i32(parent), _f64(d), _f64(u), _f64(b)
    x = np.empty_like(b)
    rc = lib().oracle_solve_batch(len(ncomp), _p(off), _p(parent), _p(d), _p(u), _p(b), _p(x), nthreads)
    if rc != OK:
        raise ValueError(f"oracle_solve_batch: status {rc}")
    return x


def matvec_batch(ncomp, parent, d, u, x):
    off = _off(ncomp)
    parent, d, u, x = _i32(parent), _f64(d), _f64(u), _f64(x)
    y = np.empty_like(x)
    lib().oracle_matvec_batch(len(ncomp), _p(off), _p(parent), _p(d), _p(u), _p(x), _p(y))
    return y


def skeel_batch(ncomp, parent, d, u, x, nthreads: int = 1):
    off = _off(ncomp)
    parent, d, u, x = _i32(parent), _f64(d), _f64(u), _f64(x)
    cond = np.empty(len(ncomp), np.float64)
    rc = lib().oracle_skeel_batch(len(ncomp), _p(off), _p(parent), _p(d), _p(u), _p(x), _p(cond), nthreads)
    if rc != OK:
        raise ValueError(f"oracle_skeel_batch: status {rc}")
    return cond


def steps_batch(ncomp, parent, s, g, a, V0, nsteps, dt, E, theta=1, nthreads: int = 1):
    """Advance V0 by nsteps implicit-Euler steps.  Returns (V, v_soma[nsteps, n_cells])."""
    off = _off(ncomp)
    parent, s, g, a = _i32(parent), _f64(s), _f64(g), _f64(a)
    V = _f64(V0).copy()
    vs = np.empty((nsteps, len(ncomp)), np.float64)
    rc = lib().oracle_steps_batch(len(ncomp), _p(off), _p(parent), _p(s), _p(g), _p(a), _p(V), nsteps, dt, E,
                                  int(theta), _p(vs), nthreads)
    if rc != OK:
        raise ValueError(f"oracle_steps_batch: status {rc}")
    return V, vs


def adjoint_batch(ncomp, parent, s, g, a, V0, target, nsteps, dt, E, theta=1, nthreads: int = 1):
    """Loss per cell and dL/dg, dL/da (per compartment; a[first of cell] unused)."""
    off = _off(ncomp)
    parent, s, g, a, V0, target = _i32(parent), _f64(s), _f64(g), _f64(a), _f64(V0), _f64(target)
    loss = np.empty(len(ncomp), np.float64)
    gg = np.empty_like(s)
    ga = np.empty_like(s)
    rc = lib().oracle_adjoint_batch(len(ncomp), _p(off), _p(parent), _p(s), _p(g), _p(a), _p(V0), _p(target),
                                    nsteps, dt, E, int(theta), _p(loss), _p(gg), _p(ga), nthreads)
    if rc != OK:
        raise ValueError(f"oracle_adjoint_batch: status {rc}")
    return loss, gg, ga
