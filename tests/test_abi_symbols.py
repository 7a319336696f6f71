"""The C-ABI library loads without a GPU and exports every entry point that
include/hines.h declares; argument errors come back as status codes."""
import ctypes
import os
import re
import subprocess

import numpy as np

from paper_1810_12742_gb300 import hines as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hines.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hines_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(H.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = H.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", H._LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hines_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_status_strings():
    for code in range(8):
        assert H.status_string(code) not in ("", "unknown status")
    assert H.status_string(99) == "unknown status"


def test_argument_errors_without_gpu():
    L = H.lib()
    h = ctypes.c_void_p()
    nc = np.array([2], np.int32)
    pa = np.array([-1, 0], np.int32)
    assert L.hines_plan_create(None, 1, nc.ctypes.data_as(ctypes.c_void_p), pa.ctypes.data_as(ctypes.c_void_p),
                               None) == H.HINES_ERR_INVALID_ARG
    opts = H.PlanOpts(1, 0, 0)
    opts.reserved[0] = 1
    assert L.hines_plan_create(ctypes.byref(h), 1, nc.ctypes.data_as(ctypes.c_void_p),
                               pa.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts)) == H.HINES_ERR_INVALID_ARG
    opts = H.PlanOpts(1, 0, 0, 0, 0, 0, 0, 0, 3)  # FP64 factor placement: 0, 1 or 2 only
    assert L.hines_plan_create(ctypes.byref(h), 1, nc.ctypes.data_as(ctypes.c_void_p),
                               pa.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts)) == H.HINES_ERR_INVALID_ARG
    opts = H.PlanOpts(1, 0, 3)  # pieces per lane: 1 or 2 only
    assert L.hines_plan_create(ctypes.byref(h), 1, nc.ctypes.data_as(ctypes.c_void_p),
                               pa.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts)) == H.HINES_ERR_INVALID_ARG
    plan = H.Plan(nc, pa, host_only=True)
    # a host-only plan refuses device work before touching CUDA
    assert L.hines_solve(plan.handle, H.HINES_F64, None, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_solve_compensated(plan.handle, None, None, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_solve_packed(plan.handle, H.HINES_F32, None, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_solve_compensated_packed(plan.handle, None, None, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pack(plan.handle, 4, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_unpack(plan.handle, 8, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_cable_step_packed(plan.handle, None, None, None, None, 0.025, -65.0, 1, None) == \
        H.HINES_ERR_INVALID_ARG
    # but its solver layout can be inspected: 2 compartments in one chunk, padded to 4 slots
    assert plan.n_packed == 4
    assert plan.export_packed().tolist() == [1, 0, -1, -1]
    # two pieces per lane: each row holds the lane's pair (the second piece absent here)
    two = H.Plan(nc, pa, host_only=True, pieces_per_lane=2)
    assert two.export_packed().tolist() == [1, -1, 0, -1]
    assert L.hines_plan_destroy(None) == H.HINES_OK


def test_pipeline_argument_errors_without_gpu():
    L = H.lib()
    h = ctypes.c_void_p()
    nc = np.array([2], np.int32)
    pa = np.array([-1, 0], np.int32)
    ncp, pap = nc.ctypes.data_as(ctypes.c_void_p), pa.ctypes.data_as(ctypes.c_void_p)
    assert L.hines_pipeline_create(None, 1, ncp, pap, 2, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pipeline_create(ctypes.byref(h), 1, ncp, pap, 0, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pipeline_create(ctypes.byref(h), -1, ncp, pap, 2, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pipeline_create(ctypes.byref(h), 1, None, pap, 2, None) == H.HINES_ERR_INVALID_ARG
    opts = H.PlanOpts(1)  # a pipeline solves: host-only plans are refused
    assert L.hines_pipeline_create(ctypes.byref(h), 1, ncp, pap, 2, ctypes.byref(opts)) == H.HINES_ERR_INVALID_ARG
    bad = np.array([-3], np.int32)
    assert L.hines_pipeline_create(ctypes.byref(h), 1, bad.ctypes.data_as(ctypes.c_void_p), pap, 2,
                                   None) == H.HINES_ERR_INVALID_ARG
    assert not h.value
    assert L.hines_pipeline_info(None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pipeline_solve_compensated(None, None, None, None, None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pipeline_status(None, None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_pipeline_destroy(None) == H.HINES_OK


def test_bounded_wait_check_argument_errors_without_gpu():
    L = H.lib()
    st = ctypes.c_int32()
    assert L.hines_check_bounded_wait(0, 0, ctypes.byref(st), None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_check_bounded_wait(1 << 17, 0, ctypes.byref(st), None) == H.HINES_ERR_INVALID_ARG
    assert L.hines_check_bounded_wait(10, 0, None, None) == H.HINES_ERR_INVALID_ARG
