"""Re-rooted plans on the GPU (Section 6, balancing the dependency tree): with
node arrays packed through the renumbering and couplings through the edge
map, the solver-layout solves and cable steps give the oracle's solution of
the caller's system; natural-layout calls are refused."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import rollout as R
from tests.test_gpu_packed import uneven_subset
from tests.test_gpu_parity import cell_rel_err, dev, zoo_batch
from tests.test_gpu_rollout import uneven_subset as uneven_steps_subset

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "comp": 1e-10}


def _solve_rerooted(plan, d, u, b, mode):
    if mode == "f64":
        xp = H.pack(plan, b)
        H.solve_packed(plan, H.pack(plan, d), H.pack_coupling(plan, u), xp)
    elif mode == "f32":
        d, u, b = (t.float() for t in (d, u, b))
        xp = H.pack(plan, b)
        H.solve_packed(plan, H.pack(plan, d), H.pack_coupling(plan, u), xp)
    else:
        d, u, b = (t.float() for t in (d, u, b))
        xp = H.solve_compensated_packed(plan, H.pack(plan, d), H.pack_coupling(plan, u), H.pack(plan, b))
    return H.unpack(plan, xp).double().cpu().numpy()


def _check(ncomp, parent, c, off, mode):
    plan = H.Plan(ncomp, parent, reroot=True)
    x = _solve_rerooted(plan, dev(c["d"]), dev(c["u"]), dev(c["b"]), mode)
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if mode != "f64" else (lambda a: a)
    ref = oracle.solve_batch(ncomp, parent, cast(c["d"]), cast(c["u"]), cast(c["b"]))
    assert cell_rel_err(x, ref, off).max() <= TOL[mode]


@pytest.mark.parametrize("mode", ["f64", "f32", "comp"])
def test_rerooted_solves_match_oracle_zoo(mode):
    ncomp, parent, c = zoo_batch(51)
    _check(ncomp, parent, c, np.concatenate(([0], np.cumsum(ncomp))), mode)


@pytest.mark.parametrize("mode", ["f64", "comp"])
def test_rerooted_solves_match_oracle_uneven(mode):
    pop = uneven_subset()
    _check(pop["ncomp"], pop["parent"], pop, pop["offsets"], mode)


@pytest.mark.parametrize("theta", [0, 1])
def test_rerooted_cable_steps_match_oracle(theta):
    w, pop = uneven_steps_subset(16, 2)
    plan = H.Plan(pop["ncomp"], pop["parent"], reroot=True)
    V = dev(pop["V0"])
    st = R.CableStepper(plan, dev(pop["s"]), dev(pop["g"]), dev(pop["u"]), V, w.dt, w.E, theta, steps=5,
                        layout="solver")
    st.replay()
    ref, _ = oracle.steps_batch(pop["ncomp"], pop["parent"], pop["s"], pop["g"], pop["a"], pop["V0"], 5, w.dt, w.E,
                             theta)
    assert cell_rel_err(st.fetch().cpu().numpy(), ref, pop["offsets"]).max() <= 1e-12


def test_rerooted_plan_refuses_natural_layout():
    ncomp, parent, c = zoo_batch(53, sizes=(5, 40))
    plan = H.Plan(ncomp, parent, reroot=True)
    d, u, b = dev(c["d"]), dev(c["u"]), dev(c["b"])
    with pytest.raises(H.HinesError) as e:
        H.solve(plan, d, u, b)
    assert e.value.code == H.HINES_ERR_INVALID_ARG
    with pytest.raises(H.HinesError):
        H.solve_compensated(plan, d.float(), u.float(), b.float())
    assert np.array_equal(b.cpu().numpy(), c["b"])  # nothing ran
