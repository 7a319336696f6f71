"""Thin ctypes binding of libhines (argument marshalling only).

Every compute step runs in the library's CUDA kernels; PyTorch only provides
device memory and the current stream.  The names follow include/hines.h.
There is no CPU fallback: loading fails loudly when libhines.so is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libhines.so")
_lock = threading.Lock()
_lib = None

HINES_OK = 0
HINES_ERR_INVALID_ARG = 1
HINES_ERR_NOT_HINES_ORDER = 2
HINES_ERR_OOM = 3
HINES_ERR_CUDA = 4
HINES_ERR_TIMEOUT = 5
HINES_WARN_REFINE = 6
HINES_ERR_DEVICE = 7
HINES_F64 = 0
HINES_F32 = 1

EXPORTS = [
    "hines_plan_create", "hines_plan_destroy", "hines_plan_layout", "hines_plan_info", "hines_plan_export",
    "hines_plan_export_tasks",
    "hines_solve", "hines_solve_compensated", "hines_solve_refine", "hines_cable_step", "hines_cable_solve", "hines_grad_du",
    "hines_cable_adjoint_step", "hines_cable_loss_seed", "hines_cable_loss_accumulate", "hines_plan_status",
    "hines_status_string",
    "hines_solve_f64_noalloc",
    "hines_plan_export_packed", "hines_pack", "hines_unpack", "hines_solve_packed", "hines_solve_compensated_packed",
    "hines_cable_step_packed", "hines_cable_solve_packed", "hines_cable_step_reuse",
    "hines_pack_coupling", "hines_plan_export_reroot",
    "hines_pipeline_create", "hines_pipeline_info", "hines_pipeline_solve_compensated", "hines_pipeline_status",
    "hines_pipeline_destroy", "hines_check_bounded_wait",
]


class HinesError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


class PlanOpts(ctypes.Structure):
    _fields_ = [("host_only", ctypes.c_int32), ("split_branches", ctypes.c_int32), ("pieces_per_lane", ctypes.c_int32),
                ("sort_by_length", ctypes.c_int32), ("pack_compartments", ctypes.c_int32),
                ("reroot", ctypes.c_int32), ("even_cuts", ctypes.c_int32), ("pack_whole", ctypes.c_int32),
                ("fp64_factor", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("n_tasks", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n_unknowns", ctypes.c_int64),
                ("n_branches", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("metadata_bytes", ctypes.c_int64), ("n_packed", ctypes.c_int64)]


def lib():
    """Load libhines.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError(f"libhines.so not built ({_LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(_LIB_PATH)
            vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
            L.hines_plan_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, ctypes.POINTER(PlanOpts)]
            L.hines_plan_destroy.argtypes = [vp]
            L.hines_plan_layout.argtypes = [vp, vp]
            L.hines_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
            L.hines_plan_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.hines_plan_export_tasks.argtypes = [vp, vp, vp, vp]
            L.hines_solve.argtypes = [vp, i32, vp, vp, vp, vp]
            L.hines_solve_refine.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp]
            L.hines_solve_compensated.argtypes = [vp, vp, vp, vp, vp, vp]
            L.hines_cable_step.argtypes = [vp, vp, vp, vp, vp, f64, f64, i32, vp]
            L.hines_cable_solve.argtypes = [vp, vp, vp, vp, vp, f64, i32, vp]
            L.hines_grad_du.argtypes = [vp, vp, vp, vp, vp, vp]
            L.hines_cable_adjoint_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, f64, f64, i32, i32, vp, vp, vp, vp]
            L.hines_cable_loss_seed.argtypes = [vp, vp, vp, vp, vp]
            L.hines_cable_loss_accumulate.argtypes = [vp, vp, vp, vp, vp]
            L.hines_plan_status.argtypes = [vp, ctypes.POINTER(i32)]
            L.hines_solve_f64_noalloc.argtypes = [ctypes.c_int64, i32, vp, vp, vp, vp, vp, vp]
            L.hines_plan_export_packed.argtypes = [vp, vp]
            L.hines_pack.argtypes = [vp, i32, vp, vp, vp]
            L.hines_unpack.argtypes = [vp, i32, vp, vp, vp]
            L.hines_pack_coupling.argtypes = [vp, i32, vp, vp, vp]
            L.hines_plan_export_reroot.argtypes = [vp, vp, vp, vp, vp]
            L.hines_solve_packed.argtypes = [vp, i32, vp, vp, vp, vp]
            L.hines_solve_compensated_packed.argtypes = [vp, vp, vp, vp, vp, vp]
            L.hines_cable_step_packed.argtypes = [vp, vp, vp, vp, vp, f64, f64, i32, vp]
            L.hines_cable_solve_packed.argtypes = [vp, vp, vp, vp, vp, f64, i32, vp]
            L.hines_cable_step_reuse.argtypes = [vp, vp, vp, vp, vp, f64, f64, i32, i32, vp]
            L.hines_status_string.argtypes = [i32]
            L.hines_pipeline_create.argtypes = [vp, i32, vp, vp, i32, vp]
            L.hines_pipeline_info.argtypes = [vp, vp, vp]
            L.hines_pipeline_solve_compensated.argtypes = [vp, vp, vp, vp, vp, vp]
            L.hines_pipeline_status.argtypes = [vp, vp]
            L.hines_pipeline_destroy.argtypes = [vp]
            L.hines_check_bounded_wait.argtypes = [i32, i32, vp, vp]
            L.hines_status_string.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name != "hines_status_string":
                    getattr(L, name).restype = i32
            _lib = L
    return _lib


_deferred = []  # plan handles whose release waits for the end of a CUDA-graph capture


def _capturing() -> bool:
    try:
        import torch
        return torch.cuda.is_available() and torch.cuda.is_current_stream_capturing()
    except Exception:
        return False


def _release_deferred():
    while _deferred and not _capturing():
        lib().hines_plan_destroy(_deferred.pop())


def status_string(code: int) -> str:
    return lib().hines_status_string(int(code)).decode()


def _check(code, where):
    if code != HINES_OK:
        raise HinesError(code, where)


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Plan:
    """Branch decomposition and schedule of a batch of cells (hines_plan_create).

    ncomp: compartments per cell; parent: the cells' parent arrays (cell-local,
    p[0] = -1, p[i] < i), concatenated.  host_only builds the schedule without
    touching the GPU (for inspection).  reroot re-roots every cell at its
    centre (Section 6); such a plan takes solver-layout arrays only (pack node
    arrays with ``pack``, couplings with ``pack_coupling``).  pieces_per_lane:
    branch pieces each warp lane owns in a chunk (1, the default, or 2).
    split_branches: False/0, True/1 (Section 6's split at the batch's level
    means) or 2 (the same at each cell's own level means).  even_cuts: cut
    long branches into near-equal pieces instead of at multiples of 8.
    pack_compartments / pack_whole: warp-task fill for the subtrees of large
    cells / for whole cells (0: as pack_compartments).  fp64_factor: where FP64
    solves and cable steps keep their factor (0 automatic, 1 natural positions,
    2 block order)."""

    def __init__(self, ncomp, parent, split_branches: bool = False, host_only: bool = False, pieces_per_lane: int = 0,
                 sort_by_length: bool = False, pack_compartments: int = 0, reroot: bool = False,
                 even_cuts: bool = False, pack_whole: int = 0, fp64_factor: int = 0):
        self._h = ctypes.c_void_p()
        _release_deferred()
        nc = np.ascontiguousarray(ncomp, np.int32)
        pa = np.ascontiguousarray(parent, np.int32)
        opts = PlanOpts(int(host_only), int(split_branches), int(pieces_per_lane), int(sort_by_length),
                        int(pack_compartments), int(reroot), int(even_cuts), int(pack_whole), int(fp64_factor))
        _check(lib().hines_plan_create(ctypes.byref(self._h), nc.size, _np_ptr(nc), _np_ptr(pa), ctypes.byref(opts)),
               "hines_plan_create")
        info = PlanInfo()
        _check(lib().hines_plan_info(self._h, ctypes.byref(info)), "hines_plan_info")
        self.n_cells = info.n_cells
        self.n_unknowns = info.n_unknowns
        self.n_branches = info.n_branches
        self.max_levels = info.max_levels
        self.n_tasks = info.n_tasks
        self.workspace_bytes = info.workspace_bytes
        self.metadata_bytes = info.metadata_bytes
        self.n_packed = info.n_packed
        self.pieces_per_lane = int(pieces_per_lane) or 1
        self.host_only = host_only
        self.rerooted = bool(reroot)
        off = np.empty(self.n_cells + 1, np.int64)
        _check(lib().hines_plan_layout(self._h, _np_ptr(off)), "hines_plan_layout")
        self.offsets = off

    @property
    def handle(self):
        return self._h

    def export(self) -> dict:
        nb = self.n_branches
        out = {k: np.empty(nb, np.int64) for k in ("first", "len", "parent_branch", "level", "cell", "order")}
        _check(lib().hines_plan_export(self._h, *(_np_ptr(out[k]) for k in
                                                  ("first", "len", "parent_branch", "level", "cell", "order"))),
               "hines_plan_export")
        return out

    def export_tasks(self) -> dict:
        out = {k: np.empty(self.n_branches, np.int64) for k in ("branch_task", "branch_kind", "task_order")}
        _check(lib().hines_plan_export_tasks(self._h, _np_ptr(out["branch_task"]), _np_ptr(out["branch_kind"]),
                                             _np_ptr(out["task_order"])), "hines_plan_export_tasks")
        return out

    def export_packed(self) -> np.ndarray:
        """Natural index held by each solver-layout slot (-1: padding)."""
        out = np.empty(self.n_packed, np.int64)
        _check(lib().hines_plan_export_packed(self._h, _np_ptr(out)), "hines_plan_export_packed")
        return out

    def export_reroot(self) -> dict:
        """The re-rooting of a plan made with reroot=True: parent (re-rooted
        cell-local parent arrays), perm and edge (caller's index of each
        re-rooted compartment and of its coupling, -1 at a root), centre."""
        out = {"parent": np.empty(self.n_unknowns, np.int32), "perm": np.empty(self.n_unknowns, np.int64),
               "edge": np.empty(self.n_unknowns, np.int64), "centre": np.empty(self.n_cells, np.int32)}
        _check(lib().hines_plan_export_reroot(self._h, *(_np_ptr(out[k]) for k in ("parent", "perm", "edge",
                                                                                   "centre"))),
               "hines_plan_export_reroot")
        return out

    def status(self) -> int:
        st = ctypes.c_int32(0)
        _check(lib().hines_plan_status(self._h, ctypes.byref(st)), "hines_plan_status")
        return st.value

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()
            if _capturing():
                # destroying synchronises the device, which would invalidate a
                # CUDA-graph capture in progress: release it after the capture
                _deferred.append(h)
            else:
                lib().hines_plan_destroy(h)
        _release_deferred()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# torch-facing calls (device tensors, current stream)
# ----------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dptr(t, dtype, n, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected contiguous {dtype} with {n} elements, got {t.dtype} {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def solve(plan: Plan, d, u, b):
    """In place: b <- A^{-1} b for every cell (FP64 or FP32 by the tensors' dtype)."""
    torch = _torch()
    n = plan.n_unknowns
    if b.dtype == torch.float64:
        dt, code = torch.float64, HINES_F64
    elif b.dtype == torch.float32:
        dt, code = torch.float32, HINES_F32
    else:
        raise ValueError("b must be float64 or float32")
    _check(lib().hines_solve(plan.handle, code, _dptr(d, dt, n, "d"), _dptr(u, dt, n, "u"), _dptr(b, dt, n, "b"),
                             _stream()), "hines_solve")
    return b


def solve_compensated(plan: Plan, d, u, b, x=None):
    """FP32 inputs, double-float (compensated FP32) elimination, FP64 solution x."""
    torch = _torch()
    n = plan.n_unknowns
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=b.device)
    _check(lib().hines_solve_compensated(plan.handle, _dptr(d, torch.float32, n, "d"), _dptr(u, torch.float32, n, "u"),
                                         _dptr(b, torch.float32, n, "b"), _dptr(x, torch.float64, n, "x"), _stream()),
           "hines_solve_compensated")
    return x


def _pptr(t, dtype, n, name):
    """Pointer to a solver-layout tensor (n_packed elements, 16-byte aligned)."""
    p = _dptr(t, dtype, n, name)
    if p.value and p.value % 16:
        raise ValueError(f"{name}: solver-layout arrays must be 16-byte aligned")
    return p


def pack(plan: Plan, natural, packed=None):
    """Natural-layout tensor (float32 or float64) -> solver layout."""
    torch = _torch()
    if packed is None:
        packed = torch.empty(plan.n_packed, dtype=natural.dtype, device=natural.device)
    eb = natural.element_size()
    _check(lib().hines_pack(plan.handle, eb, _dptr(natural, natural.dtype, plan.n_unknowns, "natural"),
                            _pptr(packed, natural.dtype, plan.n_packed, "packed"), _stream()), "hines_pack")
    return packed


def pack_coupling(plan: Plan, natural, packed=None):
    """Natural-layout coupling array u -> solver layout (hines_pack_coupling:
    through the edge map on a re-rooted plan, else the same as pack)."""
    torch = _torch()
    if packed is None:
        packed = torch.empty(plan.n_packed, dtype=natural.dtype, device=natural.device)
    eb = natural.element_size()
    _check(lib().hines_pack_coupling(plan.handle, eb, _dptr(natural, natural.dtype, plan.n_unknowns, "natural"),
                                     _pptr(packed, natural.dtype, plan.n_packed, "packed"), _stream()),
           "hines_pack_coupling")
    return packed


def unpack(plan: Plan, packed, natural=None):
    """Solver-layout tensor -> natural layout."""
    torch = _torch()
    if natural is None:
        natural = torch.empty(plan.n_unknowns, dtype=packed.dtype, device=packed.device)
    eb = packed.element_size()
    _check(lib().hines_unpack(plan.handle, eb, _pptr(packed, packed.dtype, plan.n_packed, "packed"),
                              _dptr(natural, packed.dtype, plan.n_unknowns, "natural"), _stream()), "hines_unpack")
    return natural


def solve_packed(plan: Plan, d, u, b):
    """hines_solve on solver-layout tensors (float64 or float32), in place in b."""
    torch = _torch()
    dt = b.dtype
    code = HINES_F64 if dt == torch.float64 else HINES_F32
    n = plan.n_packed
    _check(lib().hines_solve_packed(plan.handle, code, _pptr(d, dt, n, "d"), _pptr(u, dt, n, "u"),
                                    _pptr(b, dt, n, "b"), _stream()), "hines_solve_packed")
    return b


def solve_compensated_packed(plan: Plan, d, u, b, x=None):
    """hines_solve_compensated on solver-layout tensors; x float64 in the solver layout."""
    torch = _torch()
    n = plan.n_packed
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=b.device)
    _check(lib().hines_solve_compensated_packed(plan.handle, _pptr(d, torch.float32, n, "d"),
                                                _pptr(u, torch.float32, n, "u"), _pptr(b, torch.float32, n, "b"),
                                                _pptr(x, torch.float64, n, "x"), _stream()),
           "hines_solve_compensated_packed")
    return x


def cable_step_packed(plan: Plan, s, g, u, V, dt: float, E: float, theta: int = 1):
    """hines_cable_step on solver-layout float64 tensors (V in place)."""
    torch = _torch()
    n = plan.n_packed
    _check(lib().hines_cable_step_packed(plan.handle, _pptr(s, torch.float64, n, "s"), _pptr(g, torch.float64, n, "g"),
                                         _pptr(u, torch.float64, n, "u"), _pptr(V, torch.float64, n, "V"),
                                         float(dt), float(E), int(theta), _stream()), "hines_cable_step_packed")
    return V


def cable_step_reuse(plan: Plan, s, g, u, V, dt: float, E: float, theta: int = 1, solver_layout: bool = False):
    """hines_cable_step_reuse: a cable step with the factor of the last full
    step on this plan (same s, g, u, dt, theta and layout); V in place."""
    torch = _torch()
    n = plan.n_packed if solver_layout else plan.n_unknowns
    ptr = _pptr if solver_layout else _dptr
    _check(lib().hines_cable_step_reuse(plan.handle, ptr(s, torch.float64, n, "s"), ptr(g, torch.float64, n, "g"),
                                        ptr(u, torch.float64, n, "u"), ptr(V, torch.float64, n, "V"), float(dt),
                                        float(E), int(theta), int(bool(solver_layout)), _stream()),
           "hines_cable_step_reuse")
    return V


def cable_solve_packed(plan: Plan, s, g, u, y, dt: float, theta: int = 1):
    """hines_cable_solve on solver-layout float64 tensors (y in place)."""
    torch = _torch()
    n = plan.n_packed
    _check(lib().hines_cable_solve_packed(plan.handle, _pptr(s, torch.float64, n, "s"), _pptr(g, torch.float64, n, "g"),
                                          _pptr(u, torch.float64, n, "u"), _pptr(y, torch.float64, n, "y"),
                                          float(dt), int(theta), _stream()), "hines_cable_solve_packed")
    return y


def solve_refine(plan: Plan, d, u, b, x=None, steps: int = 2, relres=None):
    """FP32 elimination + iterative refinement (residual to FP64 accuracy from
    error-free FP32 products, fused with the correction's elimination);
    returns x (float64)."""
    torch = _torch()
    n = plan.n_unknowns
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=b.device)
    rr = ctypes.c_void_p(0) if relres is None else _dptr(relres, torch.float64, plan.n_cells, "relres")
    _check(lib().hines_solve_refine(plan.handle, _dptr(d, torch.float32, n, "d"), _dptr(u, torch.float32, n, "u"),
                                    _dptr(b, torch.float32, n, "b"), _dptr(x, torch.float64, n, "x"), int(steps), rr,
                                    _stream()), "hines_solve_refine")
    return x


def cable_step(plan: Plan, s, g, u, V, dt: float, E: float, theta: int = 1):
    """One fused rebuild + solve step of the passive cable; V advanced in place."""
    torch = _torch()
    n = plan.n_unknowns
    f = torch.float64
    _check(lib().hines_cable_step(plan.handle, _dptr(s, f, n, "s"), _dptr(g, f, n, "g"), _dptr(u, f, n, "u"),
                                  _dptr(V, f, n, "V"), float(dt), float(E), int(theta), _stream()),
           "hines_cable_step")
    return V


def cable_solve(plan: Plan, s, g, u, y, dt: float, theta: int = 1):
    torch = _torch()
    n = plan.n_unknowns
    f = torch.float64
    _check(lib().hines_cable_solve(plan.handle, _dptr(s, f, n, "s"), _dptr(g, f, n, "g"), _dptr(u, f, n, "u"),
                                   _dptr(y, f, n, "y"), float(dt), int(theta), _stream()), "hines_cable_solve")
    return y


def grad_du(plan: Plan, lam, x, grad_d=None, grad_u=None):
    torch = _torch()
    n = plan.n_unknowns
    f = torch.float64
    grad_d = torch.empty_like(x) if grad_d is None else grad_d
    grad_u = torch.empty_like(x) if grad_u is None else grad_u
    _check(lib().hines_grad_du(plan.handle, _dptr(lam, f, n, "lambda"), _dptr(x, f, n, "x"),
                               _dptr(grad_d, f, n, "grad_d"), _dptr(grad_u, f, n, "grad_u"), _stream()),
           "hines_grad_du")
    return grad_d, grad_u


def cable_adjoint_step(plan: Plan, lam, V_k, V_km1, s, g, target, dt, E, theta, add_loss_term, grad_g, grad_a, vbar):
    torch = _torch()
    n = plan.n_unknowns
    f = torch.float64
    tg = _dptr(target, f, plan.n_cells, "target")
    _check(lib().hines_cable_adjoint_step(plan.handle, _dptr(lam, f, n, "lambda"), _dptr(V_k, f, n, "V_k"),
                                          _dptr(V_km1, f, n, "V_km1"), _dptr(s, f, n, "s"), _dptr(g, f, n, "g"), tg,
                                          float(dt), float(E), int(theta), int(add_loss_term),
                                          _dptr(grad_g, f, n, "grad_g"), _dptr(grad_a, f, n, "grad_a"),
                                          _dptr(vbar, f, n, "vbar"), _stream()), "hines_cable_adjoint_step")


def cable_loss_seed(plan: Plan, V, target, vbar):
    torch = _torch()
    n = plan.n_unknowns
    f = torch.float64
    _check(lib().hines_cable_loss_seed(plan.handle, _dptr(V, f, n, "V"), _dptr(target, f, plan.n_cells, "target"),
                                       _dptr(vbar, f, n, "vbar"), _stream()), "hines_cable_loss_seed")


class HostPipeline:
    """hines_pipeline_*: the compensated solve from host arrays, with the
    transfers overlapped.  The library cuts the batch into ``pieces`` runs of
    consecutive cells of about equal size, each with its own plan and device
    buffers, and per run overlaps the host-to-device copies, the solve and the
    copy back on three internal streams.  ``solve_compensated`` takes CPU
    tensors in the natural layout of the whole batch (pinned, for the
    overlap) and enqueues the work after the current stream, which then waits
    for all of it.  plan_options go to every run's plan."""

    def __init__(self, ncomp, parent, pieces: int = 8, **plan_options):
        self._h = ctypes.c_void_p()
        nc = np.ascontiguousarray(ncomp, np.int32)
        pa = np.ascontiguousarray(parent, np.int32)
        o = dict(host_only=False, split_branches=0, pieces_per_lane=0, sort_by_length=False, pack_compartments=0,
                 reroot=False, even_cuts=False, pack_whole=0, fp64_factor=0)
        unknown = set(plan_options) - set(o)
        if unknown:
            raise TypeError(f"unknown plan options: {sorted(unknown)}")
        o.update(plan_options)
        opts = PlanOpts(int(o["host_only"]), int(o["split_branches"]), int(o["pieces_per_lane"]),
                        int(o["sort_by_length"]), int(o["pack_compartments"]), int(o["reroot"]),
                        int(o["even_cuts"]), int(o["pack_whole"]), int(o["fp64_factor"]))
        _check(lib().hines_pipeline_create(ctypes.byref(self._h), nc.size, _np_ptr(nc), _np_ptr(pa), int(pieces),
                                           ctypes.byref(opts)), "hines_pipeline_create")
        npieces, n = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().hines_pipeline_info(self._h, ctypes.byref(npieces), ctypes.byref(n)), "hines_pipeline_info")
        self.pieces, self.n_unknowns = npieces.value, n.value

    def solve_compensated(self, d, u, b, x):
        torch = _torch()
        n = self.n_unknowns
        _check(lib().hines_pipeline_solve_compensated(self._h, _hptr(d, torch.float32, n, "d"),
                                                      _hptr(u, torch.float32, n, "u"),
                                                      _hptr(b, torch.float32, n, "b"),
                                                      _hptr(x, torch.float64, n, "x"), _stream()),
               "hines_pipeline_solve_compensated")
        return x

    def status(self) -> int:
        s = ctypes.c_int32()
        _check(lib().hines_pipeline_status(self._h, ctypes.byref(s)), "hines_pipeline_status")
        return s.value

    def close(self):
        if self._h:
            lib().hines_pipeline_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_bounded_wait(polls: int, arrive: bool = False):
    """hines_check_bounded_wait: (status, elapsed ns) of a barrier wait that
    runs out after `polls` polls (arrive=False) or completes (arrive=True)."""
    st, ns = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().hines_check_bounded_wait(int(polls), int(bool(arrive)), ctypes.byref(st), ctypes.byref(ns)),
           "hines_check_bounded_wait")
    return st.value, ns.value


def _hptr(t, dtype, n, name):
    """Pointer to a contiguous CPU tensor (host memory)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name}: expected a CPU tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected contiguous {dtype} with {n} elements, got {t.dtype} {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())
