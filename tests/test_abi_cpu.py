"""The C-ABI library loads and exports every entry point of include/lbm.h.

These tests need no GPU: they build the library (nvcc cross-compiles for
sm_103a), load it, and exercise only host-side calls (handle creation and
argument checks), which allocate no device memory.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1108_0786_gb300 import _build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return re.findall(r"^\s*(?:int|long long|const char \*)\s*(lbm_\w+)\s*\(", hdr, re.M)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lbm.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbm.EXPORTED)


def test_only_the_c_abi_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    text_syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert text_syms == set(declared_symbols())


def test_host_side_calls_without_a_device(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(16, 16, 16, 1.0, 7, ctypes.byref(h)) == 0
    p = np.array([8.0, 8.0, 8.0])
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.lbm_add_body(h, 0, 2.0, 0.0, 10.0, p.ctypes.data_as(dp), None) == 0
    assert lib.lbm_add_body(h, 1, 1.5, 3.0, 12.0, p.ctypes.data_as(dp), None) == 1
    assert lib.lbm_add_spring(h, 0, 1, 0.01, 5.0, 0.001) == 0
    assert lib.lbm_add_spring(h, 0, 0, 0.01, 5.0, 0.001) == lbm.E_ARG
    assert lib.lbm_set_drive(h, 0, 1e-4, 1 / 400, 0.0) == 0
    assert lib.lbm_set_drive(h, 7, 1e-4, 1 / 400, 0.0) == lbm.E_ARG
    assert lib.lbm_add_body(h, 0, -1.0, 0.0, 10.0, p.ctypes.data_as(dp), None) == lbm.E_ARG
    out = np.zeros(26)
    assert lib.lbm_get_bodies(h, out.ctypes.data_as(dp)) == 0
    assert np.array_equal(out[:3], p) and out[3] == 1.0
    # before the first step an asynchronous read completes at once (ticket -1)
    out2 = np.zeros(26)
    t = ctypes.c_longlong(7)
    lib.lbm_get_bodies_async.argtypes = [ctypes.c_void_p, dp, ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_wait_ticket.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    assert lib.lbm_get_bodies_async(h, out2.ctypes.data_as(dp), ctypes.byref(t)) == 0
    assert t.value == -1 and np.array_equal(out2, out)
    assert lib.lbm_wait_ticket(h, -1) == 0
    assert lib.lbm_wait_ticket(h, 0) == lbm.E_ARG          # never issued
    # remap, bulk, boundary, links, drive and spring loads, force + integrate
    assert lib.lbm_kernels_per_step(h) == 6
    assert lib.lbm_bytes_per_cell(h) == 2 * 19 * 4 + 1
    assert lib.lbm_destroy(h) == 0


@pytest.mark.parametrize("args", [(0, 8, 8, 1.0, 7), (8, 8, 8, 0.5, 7), (8, 8, 8, 1.0, 9)])
def test_create_rejects_bad_arguments(lib, args):
    h = ctypes.c_void_p()
    assert lib.lbm_create(*args, ctypes.byref(h)) == lbm.E_ARG


def test_tune_accepts_only_compiled_shapes(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(16, 8, 8, 1.0, 7, ctypes.byref(h)) == 0
    assert lib.lbm_tune(h, 2, 4) == 0
    assert lib.lbm_tune(h, 2, 7) == lbm.E_ARG
    assert lib.lbm_tune(h, 3, 0) == lbm.E_ARG          # 16 is not a multiple of 3
    assert lib.lbm_tune(h, 0, 0) == 0
    lib.lbm_destroy(h)


def test_bytes_per_cell_by_precision(lib):
    for prec, es in ((lbm.PREC_F64, 8), (lbm.PREC_F32, 4), (lbm.PREC_F16, 2), (lbm.PREC_BF16, 2)):
        h = ctypes.c_void_p()
        assert lib.lbm_create_ex(16, 8, 8, 1.0, 7, prec, None, 0, ctypes.byref(h)) == 0
        assert lib.lbm_bytes_per_cell(h) == 2 * 19 * es + 1
        lib.lbm_destroy(h)


def test_bodies_wider_than_a_periodic_period_are_rejected(lib):
    """A capsule of radius 1.5 and length 3 has a remap cube of side
    2 (ceil(3) + 1 + 3) + 1 = 15: a periodic axis of 14 cells would make the
    per-step scans visit cells twice, so the body is refused; walls on that
    axis, or no fluid, lift the rule."""
    dp = ctypes.POINTER(ctypes.c_double)
    p = np.array([7.0, 7.5, 7.5])
    for dims, bc, options, want in (((14, 15, 15), 7, 0, lbm.E_ARG), ((15, 14, 15), 7, 0, lbm.E_ARG),
                                    ((15, 15, 14), 7, 0, lbm.E_ARG), ((15, 15, 15), 7, 0, 0),
                                    ((14, 15, 15), 6, 0, 0), ((14, 14, 14), 7, lbm.OPT_NO_FLUID, 0)):
        h = ctypes.c_void_p()
        assert lib.lbm_create_ex(*dims, 1.0, bc, lbm.PREC_F32, None, options, ctypes.byref(h)) == 0
        assert lib.lbm_add_body(h, 1, 1.5, 3.0, 12.0, p.ctypes.data_as(dp), None) == want, (dims, bc, options)
        if want:
            assert b"remap cube" in lib.lbm_last_error(h)
        lib.lbm_destroy(h)


def test_debug_knobs_take_only_their_values_before_the_first_step(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(16, 16, 16, 1.0, 7, ctypes.byref(h)) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_EXPIRE_WAITS, 1) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_EXPIRE_WAITS, 0) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_EXPIRE_WAITS, 2) == lbm.E_ARG
    assert lib.lbm_debug_set(h, lbm.DEBUG_CELL_LIST_CAP, 8) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_CELL_LIST_CAP, -1) == lbm.E_ARG
    assert lib.lbm_debug_set(h, lbm.DEBUG_ADJOINT_SERIAL, 1) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_ADJOINT_SERIAL, 0) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_ADJOINT_SERIAL, 2) == lbm.E_ARG
    assert lib.lbm_debug_set(h, lbm.DEBUG_NO_PDL, 1) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_NO_PDL, 0) == 0
    assert lib.lbm_debug_set(h, lbm.DEBUG_NO_PDL, -1) == lbm.E_ARG
    assert lib.lbm_debug_set(h, 99, 0) == lbm.E_ARG
    assert lib.lbm_destroy(h) == 0
