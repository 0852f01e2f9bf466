"""The momentum-exchange entry point that allocates no device memory.

``lbm_momentum_exchange_static`` serves callers that cannot call cudaMalloc
(their device memory sits in a pool of their own, or they must avoid the
device-wide synchronisation of cudaMalloc / cudaFree).  It takes the
populations, the obstacle-cell field and the body states of a step from the
caller and keeps its partial sums in a fixed-size static device array.

Here its output is compared with the forces the regular step reports
(``lbm_get_forces``) on two calls in a row, and with the oracle's forces on
a periodic box shorter than the scan's cube, within the tolerance of the
other FP64 tests.  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1108_0786_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1108_0786_gb300 import _build
    _build.build()
    return torch


def scenario():
    """Walls in y, a tilted capsule and two spheres with prescribed motion."""
    sc = wl.Scenario("no-alloc", 40, 30, 36, 0.9, bc=wl.PERIODIC_X | 4)
    c, s = math.cos(0.35), math.sin(0.35)
    sc.bodies.append(wl.Body(wl.CAPSULE, 3.5, 6.0, 2000.0, (12.3, 14.6, 17.2), (c, 0.2 * s, s, 0.1)))
    sc.bodies.append(wl.Body(wl.SPHERE, 4.2, 0.0, 900.0, (29.1, 15.3, 18.4)))
    sc.bodies.append(wl.Body(wl.SPHERE, 3.0, 0.0, 500.0, (38.6, 15.1, 5.2)))   # across the x boundary
    sc.springs.append(wl.Spring(0, 1, 0.02, 17.0, 0.01))
    sc.drives.append(wl.Drive(0, 3e-3, 1 / 60.0, 0.0))
    sc.drives.append(wl.Drive(1, -3e-3, 1 / 60.0, 0.0))
    return sc


def half_width(sc):
    return max(math.ceil(b.radius + 0.5 * b.length) for b in sc.bodies) + 2


def static_forces(torch, lib, pop, flags, states, sc, hw):
    bodies = torch.tensor(np.asarray(states), dtype=torch.float64, device="cuda")
    out = torch.full((len(sc.bodies), 6), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.lbm_momentum_exchange_static(
        ctypes.c_void_p(pop.data_ptr()), ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(bodies.data_ptr()),
        len(sc.bodies), sc.nx, sc.ny, sc.nz, sc.bc, hw, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(stream))
    assert rc == lbm.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def call_static(torch, lib, lat, sc, states):
    C = sc.cells
    pop = torch.empty((19, C), dtype=torch.float64, device="cuda")
    flags = torch.empty(C, dtype=torch.uint8, device="cuda")
    lat.field_device(lbm.FIELD_POP, pop, lbm.DTYPE_F64)
    lat.field_device(lbm.FIELD_FLAGS, flags, lbm.DTYPE_U8)
    return static_forces(torch, lib, pop, flags, states, sc, half_width(sc))


def test_static_scratch_forces_match_the_step_forces_on_two_calls(torch_cuda):
    torch = torch_cuda
    lib = lbm.load_library()
    sc = scenario()
    lat = lbm.from_scenario(sc, precision="f64")
    for b, v, w in ((0, (0.02, -0.01, 0.005), (0.002, -0.001, 0.003)), (1, (-0.015, 0.01, 0.0), (0, 0, 0.001)),
                    (2, (0.0, 0.01, -0.02), (0.001, 0.0, 0.0))):
        s = lat.bodies()[b].copy()
        s[7:10] = v
        s[10:13] = w
        lat.set_body_state(b, s)
    lat.step(25)
    for _ in range(2):
        states = lat.bodies()          # the state the next step maps and sums with
        lat.step(1)
        ref = lat.forces()
        got = call_static(torch, lib, lat, sc, states)
        assert np.isfinite(got).all()
        assert np.abs(ref).max() > 1e-6
        assert np.abs(got - ref).max() < 1e-12 + 1e-10 * np.abs(ref).max()
        lat.step(7)


def test_static_scratch_counts_each_link_once_on_short_periodic_axes(torch_cuda):
    """A 13 x 15 x 14 periodic box and a scan cube of side 19: the scan is
    cut to one period on every axis, and the forces equal the oracle's on
    the same state (the oracle's populations, map and body states)."""
    import oracle
    torch = torch_cuda
    lib = lbm.load_library()
    sc = wl.Scenario("short periodic axes", 13, 15, 14, 0.9)
    c, s = math.cos(0.5), math.sin(0.5)
    sc.bodies.append(wl.Body(wl.CAPSULE, 2.2, 3.0, 300.0, (6.3, 7.6, 6.8), (c, 0.3 * s, s, 0.2)))
    ref = oracle.from_scenario(sc)
    st = ref.bodies()[0].copy()
    st[7:10] = (0.02, -0.015, 0.01)
    st[10:13] = (0.003, -0.002, 0.004)
    ref.set_body_state(0, st)
    for steps in (6, 3):
        ref.step(steps - 1)
        states = ref.bodies()                 # the state the next step maps and sums with
        ref.step(1)
        want = ref.forces()
        pop = torch.from_numpy(ref.pop().reshape(19, -1)).to("cuda")
        flags = torch.from_numpy(ref.flags().reshape(-1)).to("cuda")
        assert np.abs(want).max() > 1e-6
        for hw in (5, 9):                      # cube side 11 fits every axis; 19 fits none
            got = static_forces(torch, lib, pop, flags, states, sc, hw)
            assert np.abs(got - want).max() < 1e-12 + 1e-10 * np.abs(want).max(), hw


def test_static_scratch_rejects_sizes_beyond_its_limit(torch_cuda):
    torch = torch_cuda
    lib = lbm.load_library()
    # small real buffers: a check that stopped rejecting would read them,
    # not an arbitrary address, and fail the comparison instead
    pop = torch.zeros((19, 512), dtype=torch.float64, device="cuda")
    flags = torch.zeros(512, dtype=torch.uint8, device="cuda")
    bodies = torch.zeros((255, 13), dtype=torch.float64, device="cuda")
    out = torch.zeros((255, 6), dtype=torch.float64, device="cuda")
    p, f, b, o = (ctypes.c_void_p(t.data_ptr()) for t in (pop, flags, bodies, out))
    assert lib.lbm_momentum_exchange_static(p, f, b, 255, 8, 8, 8, 7, 4, o, None) == lbm.E_ARG
    assert lib.lbm_momentum_exchange_static(p, f, b, 2, 8, 8, 8, 7, 65, o, None) == lbm.E_ARG
    # 32 bodies with cubes of side 81 in a walled 8^3 box (walls do not cut
    # the scan): 32 * ceil(81^3 / 256) = 66432 records > 65536
    assert lib.lbm_momentum_exchange_static(p, f, b, 32, 8, 8, 8, 0, 40, o, None) == lbm.E_ARG
    assert lib.lbm_momentum_exchange_static(p, f, b, 31, 8, 8, 8, 0, 40, o, None) == lbm.OK
    assert lib.lbm_momentum_exchange_static(None, f, b, 2, 8, 8, 8, 7, 4, o, None) == lbm.E_ARG
    torch.cuda.synchronize()
    assert not out.any()             # no solid cell, no link: zero force where a call ran
