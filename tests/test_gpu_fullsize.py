"""Parity at the full workload sizes, in the launch configuration bench.py
times: the whole population is solved on the GPU and sampled cells of both
size classes are checked against the oracle one by one."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _sample(w, per_class=12, seed=3):
    cls = I.cell_classes(w)
    rng = np.random.default_rng(seed)
    picks = [rng.choice(np.nonzero(cls == k)[0], min(per_class, int((cls == k).sum())), replace=False)
             for k in range(len(w.classes))]
    return np.sort(np.concatenate(picks))


def _err(x, pop, cells, widen):
    off = pop["offsets"]
    e = 0.0
    for c in cells:
        sl = slice(off[c], off[c + 1])
        arrs = [pop[k][sl].astype(np.float32).astype(np.float64) if widen else pop[k][sl] for k in ("d", "u", "b")]
        ref = oracle.solve_batch(pop["ncomp"][c:c + 1], pop["parent"][sl], *arrs)
        e = max(e, float(np.abs(x[sl] - ref).max() / np.abs(ref).max()))
    return e


def test_uneven_population_full_size():
    w = I.WORKLOADS["uneven_mixed"]
    pop = I.population(w, margin=0.1)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    cells = _sample(w)
    f32 = {k: torch.as_tensor(pop[k].astype(np.float32)).cuda() for k in ("d", "u", "b")}
    xc = H.solve_compensated(plan, f32["d"], f32["u"], f32["b"]).cpu().numpy()
    assert _err(xc, pop, cells, True) <= 1e-10
    pk = {k: H.pack(plan, f32[k]) for k in ("d", "u", "b")}
    xp = H.unpack(plan, H.solve_compensated_packed(plan, pk["d"], pk["u"], pk["b"])).cpu().numpy()
    assert np.array_equal(xp, xc)
    del pk
    xr = H.solve_refine(plan, f32["d"], f32["u"], f32["b"], steps=2).cpu().numpy()
    assert _err(xr, pop, cells, True) <= 1e-10
    del f32
    x64 = torch.as_tensor(pop["b"]).cuda()
    H.solve(plan, torch.as_tensor(pop["d"]).cuda(), torch.as_tensor(pop["u"]).cuda(), x64)
    assert _err(x64.cpu().numpy(), pop, cells, False) <= 1e-12
    assert plan.status() == 0


def test_uniform_population_full_size_fp64():
    w = I.WORKLOADS["fp64_uniform"]
    pop = I.population(w)
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = torch.as_tensor(pop["b"]).cuda()
    H.solve(plan, torch.as_tensor(pop["d"]).cuda(), torch.as_tensor(pop["u"]).cuda(), x)
    assert _err(x.cpu().numpy(), pop, _sample(w, per_class=24), False) <= 1e-12
