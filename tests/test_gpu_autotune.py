"""The plan autotuner: it picks the fastest of its candidate options on a
synthetic system of the morphology, caches the choice, and the plan it
returns meets the solve's tolerance against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import autotune as T
from paper_1810_12742_gb300 import hines as H
from tests.test_gpu_packed import uneven_subset
from tests.test_gpu_parity import cell_rel_err, dev

pytestmark = pytest.mark.gpu


def test_tune_picks_the_fastest_and_caches(tmp_path):
    pop = uneven_subset()
    cache = str(tmp_path / "tune.json")
    cands = [dict(pack_compartments=4096), dict(pack_compartments=24576), dict(pack_compartments=24576,
                                                                              sort_by_length=True)]
    plan, rep = T.tune_plan(pop["ncomp"], pop["parent"], candidates=cands, reps=2, cache_path=cache)
    assert not rep["cached"] and rep["options"] in cands
    assert min(rep["ms"].values()) == rep["ms"][__import__("json").dumps(rep["options"], sort_keys=True)]
    plan2, rep2 = T.tune_plan(pop["ncomp"], pop["parent"], candidates=cands, cache_path=cache)
    assert rep2["cached"] and rep2["options"] == rep["options"]
    f32 = {k: pop[k].astype(np.float32) for k in ("d", "u", "b")}
    x = H.solve_compensated(plan2, *(dev(f32[k], torch.float32) for k in ("d", "u", "b"))).cpu().numpy()
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f32[k].astype(np.float64) for k in ("d", "u", "b")))
    assert cell_rel_err(x, ref, pop["offsets"]).max() <= 1e-10
    # the cached options rebuild the tuned plan: the same schedule, the same bits
    xt = H.solve_compensated(plan, *(dev(f32[k], torch.float32) for k in ("d", "u", "b"))).cpu().numpy()
    assert np.array_equal(x, xt)


def test_synthetic_system_is_diagonally_dominant():
    pop = uneven_subset()
    d, u, b = T._system(pop["ncomp"], pop["parent"])
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = b.clone()
    H.solve(plan, d, u, x)
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], d.cpu().numpy(), u.cpu().numpy(), b.cpu().numpy())
    assert cell_rel_err(x.cpu().numpy(), ref, pop["offsets"]).max() <= 1e-12
    # strict dominance: d_i exceeds the couplings of row i by s_i >= 0.01
    off = pop["offsets"]
    dn, un = d.cpu().numpy(), u.cpu().numpy()
    row = np.abs(un).copy()
    par = pop["parent"].astype(np.int64) + np.repeat(off[:-1], pop["ncomp"])
    nonroot = np.ones(dn.size, bool)
    nonroot[off[:-1][pop["ncomp"] > 0]] = False
    row[~nonroot] = 0.0
    np.add.at(row, par[nonroot], np.abs(un[nonroot]))
    assert (dn - row >= 0.01 - 1e-12).all()


def test_tune_solver_layout_with_rerooted_candidates(tmp_path):
    pop = uneven_subset()
    cands = [dict(pack_compartments=24576), dict(pack_compartments=24576, reroot=True)]
    plan, rep = T.tune_plan(pop["ncomp"], pop["parent"], layout="solver", candidates=cands, reps=2,
                            cache_path=str(tmp_path / "tune.json"))
    assert rep["options"] in cands and len(rep["ms"]) == 2
    f32 = {k: dev(pop[k].astype(np.float32), torch.float32) for k in ("d", "u", "b")}
    xp = H.solve_compensated_packed(plan, H.pack(plan, f32["d"]), H.pack_coupling(plan, f32["u"]),
                                    H.pack(plan, f32["b"]))
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"],
                             *(pop[k].astype(np.float32).astype(np.float64) for k in ("d", "u", "b")))
    assert cell_rel_err(H.unpack(plan, xp).cpu().numpy(), ref, pop["offsets"]).max() <= 1e-10
    with pytest.raises(ValueError):
        T.tune_plan(pop["ncomp"], pop["parent"], layout="natural", candidates=cands)


@pytest.mark.parametrize("solve,layout", [("compensated", "natural"), ("refine", "natural"), ("cable", "solver"),
                                          ("f64", "natural")])
def test_search_tunes_every_option_and_meets_the_gate(tmp_path, solve, layout):
    """The default search visits every option of the space (per size class
    fills, lane mapping, cut rule, split, order; re-rooting in the solver
    layout), keeps the fastest, caches it, and the tuned plan still solves to
    the mode's tolerance against the oracle."""
    pop = uneven_subset()
    cache = str(tmp_path / "tune.json")
    plan, rep = T.tune_plan(pop["ncomp"], pop["parent"], solve, layout, reps=1, cache_path=cache)
    space = T.SEARCH_SPACE + (T.SOLVER_LAYOUT_SPACE if layout == "solver" else ()) + (
        T.FP64_SPACE if solve in ("f64", "cable") else ())
    assert len(rep["ms"]) >= sum(len(v) for _, v in space) - len(space)
    assert set(rep["options"]) <= {k for k, _ in space}
    assert rep["ms"][__import__("json").dumps(rep["options"], sort_keys=True)] == min(rep["ms"].values())
    again, rep2 = T.tune_plan(pop["ncomp"], pop["parent"], solve, layout, cache_path=cache)
    assert rep2["cached"] and rep2["options"] == rep["options"]
    untuned, rep3 = T.tune_plan(pop["ncomp"], pop["parent"], solve, layout, cache_path=str(tmp_path / "none.json"),
                                tune_on_miss=False)
    assert rep3["options"] is None and not rep3["cached"]
    if solve in ("compensated", "refine") and layout == "natural":
        f32 = {k: pop[k].astype(np.float32) for k in ("d", "u", "b")}
        args = [dev(f32[k], torch.float32) for k in ("d", "u", "b")]
        x = (H.solve_compensated(again, *args) if solve == "compensated"
             else H.solve_refine(again, *args, steps=1)).cpu().numpy()
        ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f32[k].astype(np.float64) for k in ("d", "u", "b")))
        assert cell_rel_err(x, ref, pop["offsets"]).max() <= 1e-10
    if solve == "f64":
        x = dev(pop["b"])
        H.solve(again, dev(pop["d"]), dev(pop["u"]), x)
        ref = oracle.solve_batch(pop["ncomp"], pop["parent"], pop["d"], pop["u"], pop["b"])
        assert cell_rel_err(x.cpu().numpy(), ref, pop["offsets"]).max() <= 1e-12
