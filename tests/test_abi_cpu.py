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


def test_every_entry_point_rejects_a_null_handle(lib):
    """Each call that takes a handle (or an ensemble) returns LBM_E_ARG for a
    null one before touching anything; destroying null is a no-op, and the
    error strings say what happened."""
    raw = ctypes.CDLL(_build.LIB)           # no argtypes: every argument marshalled as below
    hdr = open(os.path.join(ROOT, "include", "lbm.h")).read()
    decls = re.findall(r"^\s*(int|long long|const char \*)\s*(lbm_\w+)\s*\(([^;]*?)\);", hdr, re.M | re.S)
    seen = 0
    for ret, name, params in decls:
        ps = [p.strip() for p in params.replace("\n", " ").split(",")]
        if not ps[0].startswith(("lbm_t *", "lbm_ensemble_t *")):
            continue
        args = []
        for p in ps:
            if "*" in p or "[" in p or p.split()[0].endswith("_fn"):
                args.append(ctypes.c_void_p(None))
            elif p.startswith("double"):
                args.append(ctypes.c_double(0.0))
            elif p.startswith("long long"):
                args.append(ctypes.c_longlong(0))
            else:
                args.append(ctypes.c_int(0))
        f = getattr(raw, name)
        f.restype = {"int": ctypes.c_int, "long long": ctypes.c_longlong, "const char *": ctypes.c_char_p}[ret]
        r = f(*args)
        if name.endswith("_destroy"):
            assert r == 0, name
        elif ret == "const char *":
            assert r == b"null handle", name
        else:
            assert r == lbm.E_ARG, (name, r)
        seen += 1
    assert seen >= 40


def test_argument_errors_name_the_call(lib):
    """Bad arguments are refused on the host, before any device work, and
    lbm_last_error says which call refused them."""
    L = ctypes.CDLL(_build.LIB)
    L.lbm_last_error.restype = ctypes.c_char_p
    dp = ctypes.POINTER(ctypes.c_double)
    D = ctypes.c_double
    h = ctypes.c_void_p()
    assert L.lbm_create(16, 16, 16, D(1.0), 7, ctypes.byref(h)) == 0
    p = np.array([8.0, 8.0, 8.0])
    assert L.lbm_add_body(h, 0, D(2.0), D(0.0), D(10.0), p.ctypes.data_as(dp), None) == 0
    assert L.lbm_set_drive(h, 0, D(1e-4), D(0.01), D(0.0)) == 0
    cases = [
        (lambda: L.lbm_add_body(h, 0, D(2.0), D(0.0), D(10.0), None, None), b"lbm_add_body"),
        (lambda: L.lbm_set_drive_axis(h, 3, p.ctypes.data_as(dp)), b"lbm_set_drive_axis"),
        (lambda: L.lbm_set_drive_window(h, 9, D(10.0)), b"lbm_set_drive_window"),
        (lambda: L.lbm_set_body_state(h, 7, np.zeros(13).ctypes.data_as(dp)), b"lbm_set_body_state"),
        (lambda: L.lbm_set_fields(h, lbm.FIELD_POP, None, lbm.DTYPE_F64), b"lbm_set_fields"),
        (lambda: L.lbm_step(h, -1), b"lbm_step"),
        (lambda: L.lbm_get_bodies(h, None), b"lbm_get_bodies"),
        (lambda: L.lbm_get_forces(h, None), b"lbm_get_forces"),
        (lambda: L.lbm_get_fields(h, lbm.FIELD_RHO, None, lbm.DTYPE_F64), b"lbm_get_fields"),
        (lambda: L.lbm_get_fields_device(h, lbm.FIELD_RHO, None, lbm.DTYPE_F64), b"lbm_get_fields_device"),
        (lambda: L.lbm_enable_history(h, -1), b"lbm_enable_history"),
        (lambda: L.lbm_get_history(h, None, 10, None), b"lbm_get_history"),
        (lambda: L.lbm_save(h, None), b"lbm_save"),
        (lambda: L.lbm_load(h, None), b"lbm_load"),
        (lambda: L.lbm_tune(h, 2, -1), b"lbm_tune"),
        (lambda: L.lbm_autotune(h, 0, None, None), b"lbm_autotune"),
        (lambda: L.lbm_adjoint_record(h, 0, 4), b"lbm_adjoint_record"),
        (lambda: L.lbm_adjoint_backward(h, None, None, None, None, None, None, None), b"lbm_adjoint_backward"),
        (lambda: L.lbm_average_get(h, None, None), b"lbm_average_get"),
    ]
    for call, name in cases:
        assert call() == lbm.E_ARG, name
        assert L.lbm_last_error(h).startswith(name), (name, L.lbm_last_error(h))
    assert L.lbm_destroy(h) == 0
