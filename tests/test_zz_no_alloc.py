"""Allocation-free solve entry point (hines_solve_f64_noalloc), for callers
that may not allocate device memory and therefore cannot create a plan.

Called through the C-ABI with ctypes and checked against the oracle and the
plan-based FP64 solve (hines_solve) within the FP64 parity tolerance, on two
calls in a row (the second call finds the first call's values in the shared scratch
array).  This file is collected last so that a failure here stops a -x run
only after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from tests.helpers import problem, tree_zoo

pytestmark = pytest.mark.gpu


def _batch(seed):
    rng = np.random.default_rng(seed)
    trees, coef = [], {k: [] for k in ("d", "u", "b")}
    for n in (1, 2, 40, 333, 2000):
        for t in tree_zoo(rng, n).values():
            trees.append(t)
            pr = problem(t, rng)
            for k in coef:
                coef[k].append(pr[k])
    ncomp = np.array([t.size for t in trees], np.int32)
    return ncomp, np.concatenate(trees), {k: np.concatenate(v) for k, v in coef.items()}


def _noalloc(n, ncells, off, parent, d, u, b):
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return H.lib().hines_solve_f64_noalloc(n, ncells, ptr(off), ptr(parent), ptr(d), ptr(u), ptr(b), stream)


def test_noalloc_matches_plan_solve_twice():
    ncomp, parent, c = _batch(41)
    n = int(ncomp.sum())
    plan = H.Plan(ncomp, parent)
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", t)  # noqa: E731
    d, u = dev(c["d"]), dev(c["u"])
    ref = dev(c["b"])
    H.solve(plan, d, u, ref)
    off = dev(plan.offsets, torch.int64)
    par = dev(parent, torch.int32)
    exact = oracle.solve_batch(ncomp, parent, c["d"], c["u"], c["b"])
    for rep in range(2):
        x = dev(c["b"] * (1.0 + rep))
        assert _noalloc(n, len(ncomp), off, par, d, u, x) == H.HINES_OK
        torch.cuda.synchronize()
        want = ref.cpu().numpy() * (1.0 + rep)
        got = x.cpu().numpy()
        for k in range(len(ncomp)):
            sl = slice(plan.offsets[k], plan.offsets[k + 1])
            assert np.abs(got[sl] - want[sl]).max() <= 1e-12 * np.abs(want[sl]).max()
            scale = np.abs(exact[sl]).max() * (1.0 + rep)
            assert np.abs(got[sl] - exact[sl] * (1.0 + rep)).max() <= 1e-12 * scale


def test_noalloc_bad_parent_cell_is_nan_others_solved():
    """A cell whose parent array breaks Hines order comes back NaN; the cells
    around it are still solved and match the oracle."""
    ncomp, parent, c = _batch(42)
    bad = int(np.nonzero(ncomp > 5)[0][1])  # a cell of the zoo with more than five compartments
    off = np.concatenate(([0], np.cumsum(ncomp))).astype(np.int64)
    par = parent.copy()
    par[off[bad] + 2] = 5  # p[i] >= i breaks Hines order
    n = int(ncomp.sum())
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", t)  # noqa: E731
    x = dev(c["b"])
    assert _noalloc(n, len(ncomp), dev(off, torch.int64), dev(par, torch.int32), dev(c["d"]), dev(c["u"]),
                    x) == H.HINES_OK
    got = x.cpu().numpy()
    exact = oracle.solve_batch(ncomp, parent, c["d"], c["u"], c["b"])
    for k in range(len(ncomp)):
        sl = slice(off[k], off[k + 1])
        if k == bad:
            assert np.isnan(got[sl]).all()
        else:
            assert np.abs(got[sl] - exact[sl]).max() <= 1e-12 * np.abs(exact[sl]).max()


def test_noalloc_bad_offsets_leave_nan_and_empty_batch_is_ok():
    ncomp, parent, c = _batch(43)
    n = int(ncomp.sum())
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", t)  # noqa: E731
    off = np.concatenate(([0], np.cumsum(ncomp))).astype(np.int64)
    off[2], off[3] = off[3], off[2]  # not non-decreasing: two cells would overlap
    x = dev(c["b"])
    assert _noalloc(n, len(ncomp), dev(off, torch.int64), dev(parent, torch.int32), dev(c["d"]), dev(c["u"]),
                    x) == H.HINES_OK
    assert torch.isnan(x).all()
    # no cells: nothing to do, nothing touched
    y = dev(c["b"])
    assert H.lib().hines_solve_f64_noalloc(n, 0, None, None, None, None, None, None) == H.HINES_OK
    assert torch.equal(y, dev(c["b"]))
    # a valid call afterwards still solves (the validity word is rewritten by every call)
    good = np.concatenate(([0], np.cumsum(ncomp))).astype(np.int64)
    x = dev(c["b"])
    assert _noalloc(n, len(ncomp), dev(good, torch.int64), dev(parent, torch.int32), dev(c["d"]), dev(c["u"]),
                    x) == H.HINES_OK
    exact = oracle.solve_batch(ncomp, parent, c["d"], c["u"], c["b"])
    got = x.cpu().numpy()
    for k in range(len(ncomp)):
        sl = slice(good[k], good[k + 1])
        assert np.abs(got[sl] - exact[sl]).max() <= 1e-12 * np.abs(exact[sl]).max()


def test_noalloc_rejects_oversized_batch():
    big = (1 << 21) + 1
    assert H.lib().hines_solve_f64_noalloc(big, 1, None, None, None, None, None, None) == H.HINES_ERR_INVALID_ARG
