"""Solver layout (Section 5's per-chunk interleaving) through the C-ABI:
pack/unpack round trips, and solves on solver-layout arrays.  The FP64 and
FP32 solves must give bit for bit the results of the natural-layout solves
and so must the compensated solve (the arithmetic and its order are the
same; only where each value lives differs).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I
from tests.test_gpu_parity import cell_rel_err, dev, zoo_batch

pytestmark = pytest.mark.gpu


def uneven_subset():
    w = I.WORKLOADS["uneven_mixed"]
    cls = I.cell_classes(w)
    cells = np.concatenate([np.nonzero(cls == 0)[0][:40], np.nonzero(cls == 1)[0][:6]])
    return I.population(w, cells=cells, margin=0.1)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_pack_unpack_round_trip(dtype):
    ncomp, parent, c = zoo_batch(41)
    plan = H.Plan(ncomp, parent)
    a = dev(c["b"], dtype)
    pk = H.pack(plan, a)
    assert pk.numel() == plan.n_packed
    slots = plan.export_packed()
    ref = np.zeros(plan.n_packed)
    ref[slots >= 0] = a.cpu().numpy()[slots[slots >= 0]]
    assert np.array_equal(pk.cpu().numpy(), ref.astype(pk.cpu().numpy().dtype))
    back = H.unpack(plan, pk)
    assert torch.equal(back, a)


def _packed_reference(plan, host, coupling=False):
    """Every slot from the plan's exported maps: the caller's value, zero in
    padding; for couplings of a re-rooted plan, the value at the slot's edge."""
    slots = plan.export_packed()
    if coupling:
        rr = plan.export_reroot()
        inv = np.empty_like(rr["perm"])
        inv[rr["perm"]] = np.arange(rr["perm"].size)
        src = np.full(slots.size, -1, np.int64)
        src[slots >= 0] = rr["edge"][inv[slots[slots >= 0]]]
    else:
        src = slots
    ref = np.zeros(plan.n_packed, host.dtype)
    ref[src >= 0] = host[src[src >= 0]]
    return ref


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("opts", [dict(pieces_per_lane=2), dict(split_branches=1, even_cuts=True),
                                  dict(reroot=True), dict(reroot=True, pieces_per_lane=2)],
                         ids=["two_per_lane", "split_even", "rerooted", "rerooted_two_per_lane"])
@pytest.mark.parametrize("batch", ["zoo", "uneven"])
def test_pack_unpack_exact_for_every_plan_kind(dtype, opts, batch):
    """Chunk-by-chunk permutations on every kind of plan: the packed array
    equals the plan's slot map applied on the host (padding slots zero), the
    couplings of a re-rooted plan follow its edge map, and unpacking gives
    the caller's array back bit for bit."""
    if batch == "zoo":
        ncomp, parent, c = zoo_batch(43)
        b = c["b"]
    else:
        pop = uneven_subset()
        ncomp, parent, b = pop["ncomp"], pop["parent"], pop["b"]
    plan = H.Plan(ncomp, parent, **opts)
    a = dev(b, dtype)
    host = a.cpu().numpy()
    pk = H.pack(plan, a)
    assert np.array_equal(pk.cpu().numpy(), _packed_reference(plan, host))
    assert torch.equal(H.unpack(plan, pk), a)
    pc = H.pack_coupling(plan, a).cpu().numpy()
    assert np.array_equal(pc, _packed_reference(plan, host, coupling=bool(opts.get("reroot"))))
    assert plan.status() == 0


def _natural_and_packed(plan, d, u, b, mode):
    if mode == "f64":
        x = b.clone()
        H.solve(plan, d, u, x)
        xp = H.pack(plan, b)
        H.solve_packed(plan, H.pack(plan, d), H.pack(plan, u), xp)
        return x, H.unpack(plan, xp)
    if mode == "f32":
        d, u, b = (t.float() for t in (d, u, b))
        x = b.clone()
        H.solve(plan, d, u, x)
        xp = H.pack(plan, b)
        H.solve_packed(plan, H.pack(plan, d), H.pack(plan, u), xp)
        return x, H.unpack(plan, xp)
    d, u, b = (t.float() for t in (d, u, b))
    x = H.solve_compensated(plan, d, u, b)
    xp = H.solve_compensated_packed(plan, H.pack(plan, d), H.pack(plan, u), H.pack(plan, b))
    return x, H.unpack(plan, xp)


def _same(x, xp, mode, off):
    assert torch.equal(x, xp), (mode, cell_rel_err(xp.double().cpu().numpy(), x.double().cpu().numpy(), off).max())


@pytest.mark.parametrize("mode", ["f64", "f32", "comp"])
@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("per_lane", [1, 2])
def test_packed_solves_equal_natural_zoo(mode, split, per_lane):
    ncomp, parent, c = zoo_batch(43)
    plan = H.Plan(ncomp, parent, split_branches=split, pieces_per_lane=per_lane)
    x, xp = _natural_and_packed(plan, dev(c["d"]), dev(c["u"]), dev(c["b"]), mode)
    _same(x, xp, mode, np.concatenate(([0], np.cumsum(ncomp))))
    widen = mode != "f64"
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if widen else (lambda a: a)
    ref = oracle.solve_batch(ncomp, parent, cast(c["d"]), cast(c["u"]), cast(c["b"]))
    tol = {"f64": 1e-12, "f32": 1e-5, "comp": 1e-10}[mode]
    assert cell_rel_err(xp.double().cpu().numpy(), ref, np.concatenate(([0], np.cumsum(ncomp)))).max() <= tol


@pytest.mark.parametrize("mode", ["f64", "f32", "comp"])
@pytest.mark.parametrize("pack", [0, -1])
@pytest.mark.parametrize("per_lane", [1, 2])
def test_packed_solves_equal_natural_uneven(mode, pack, per_lane):
    pop = uneven_subset()
    plan = H.Plan(pop["ncomp"], pop["parent"], pack_compartments=pack, pieces_per_lane=per_lane)
    x, xp = _natural_and_packed(plan, dev(pop["d"]), dev(pop["u"]), dev(pop["b"]), mode)
    _same(x, xp, mode, pop["offsets"])


def test_packed_inputs_not_modified_and_repeatable():
    ncomp, parent, c = zoo_batch(47)
    plan = H.Plan(ncomp, parent)
    d, u, b = (H.pack(plan, dev(c[k], torch.float32)) for k in ("d", "u", "b"))
    d0, u0, b0 = d.clone(), u.clone(), b.clone()
    x1 = H.solve_compensated_packed(plan, d, u, b)
    x2 = H.solve_compensated_packed(plan, d, u, b)
    assert torch.equal(d, d0) and torch.equal(u, u0) and torch.equal(b, b0)
    real = torch.as_tensor(plan.export_packed() >= 0, device="cuda")
    assert torch.equal(x1[real], x2[real])


def test_packed_misaligned_rejected():
    ncomp, parent, c = zoo_batch(49, sizes=(17, 64))
    plan = H.Plan(ncomp, parent)
    buf = torch.zeros(plan.n_packed + 1, dtype=torch.float32, device="cuda")
    d = buf[1:]  # 4-byte offset: not 16-byte aligned
    ok = H.pack(plan, dev(c["d"], torch.float32))
    with pytest.raises(ValueError):
        H.solve_compensated_packed(plan, d, ok, ok)
    x = torch.empty(plan.n_packed, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    code = H.lib().hines_solve_compensated_packed(plan.handle, vp(d.data_ptr()), vp(ok.data_ptr()),
                                                  vp(ok.data_ptr()), vp(x.data_ptr()), vp(0))
    assert code == 1  # HINES_ERR_INVALID_ARG, nothing launched


def test_host_pipeline_equals_device_solve():
    """The overlapped host-array pipeline (pieces with their own plans) gives
    the whole-batch compensated solve to rounding: cells are independent, but
    each piece's plan cuts long branches at multiples of 8 of its own buffers,
    so the pieces' chains (and their roundings) can differ from the whole
    batch's.  Both stay within the FP32-input gate of the oracle."""
    pop = uneven_subset()
    plan = H.Plan(pop["ncomp"], pop["parent"])
    f32 = {k: pop[k].astype(np.float32) for k in ("d", "u", "b")}
    x = H.solve_compensated(plan, *(dev(f32[k], torch.float32) for k in ("d", "u", "b"))).cpu().numpy()
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], *(f32[k].astype(np.float64) for k in ("d", "u", "b")))
    host = {k: torch.as_tensor(f32[k]).pin_memory() for k in ("d", "u", "b")}
    xh = torch.empty(plan.n_unknowns, dtype=torch.float64).pin_memory()
    for pieces in (1, 3, 7):
        pipe = H.HostPipeline(pop["ncomp"], pop["parent"], pieces=pieces)
        xh.zero_()
        pipe.solve_compensated(host["d"], host["u"], host["b"], xh)
        torch.cuda.synchronize()
        got = xh.numpy()
        if pieces == 1:
            assert np.array_equal(got, x)  # one piece: the same plan, the same arithmetic
        assert cell_rel_err(got, x, plan.offsets).max() <= 1e-12
        assert cell_rel_err(got, ref, plan.offsets).max() <= 1e-10
        assert pipe.status() == 0
    # pageable host arrays: the copies complete without overlap, same results
    pipe = H.HostPipeline(pop["ncomp"], pop["parent"], pieces=3)
    xp = torch.zeros(plan.n_unknowns, dtype=torch.float64)
    pipe.solve_compensated(*(torch.as_tensor(f32[k]) for k in ("d", "u", "b")), xp)
    torch.cuda.synchronize()
    pipe.solve_compensated(host["d"], host["u"], host["b"], xh)
    torch.cuda.synchronize()
    assert np.array_equal(xp.numpy(), xh.numpy())
    pipe.close()
