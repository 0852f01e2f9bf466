"""Failure detection on the GPU: every latched status bit the library can
raise is driven through the public API, and the error surfaces at the next
synchronising call as its LBM_E_* code.

No test faults, traps or hangs the GPU.  The failing situations are made on
the host: populations set to NaN, a body state set faster than
LBM_MAX_BODY_STEP, a cell-list capacity too small for the bodies
(LBM_DEBUG_CELL_LIST_CAP); and, for the bounded waits of the row-staged bulk
kernel, a test switch (LBM_DEBUG_EXPIRE_WAITS) that makes each block's first
wait be on a barrier nothing completes, bounded by ~2^16 cycles.
Overlapping bodies and a body crossing a wall are driven in
test_gpu_parity.py.  Each handle is stepped
only as far as the step that latches the error (a step after a non-finite
state would map bodies from non-finite positions), and a fresh handle then
runs a correct step on the same context.
"""
import numpy as np
import pytest

from paper_1108_0786_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1108_0786_gb300 import _build
    _build.build()
    return torch


def swimmer(n=32, precision="f32"):
    sc = wl.Scenario("failure", n, n, n, 1.0)
    wl.add_swimmer(sc, (n / 2 + 0.3, n / 2 - 0.2, n / 2 + 0.1), (1.0, 0.0, 0.0, 0.0), (wl.SPHERE,) * 3, 3.0, 0.0,
                   9.0, 0.01, 0.005, 1e-3, 100.0, density=2.0)
    return lbm.from_scenario(sc, precision=precision)


def expect_error(lat, code):
    with pytest.raises(lbm.LbmError) as ei:
        lat.sync()
    assert ei.value.code == code, (ei.value.code, str(ei.value))
    # latched: the next synchronising call reports it again
    with pytest.raises(lbm.LbmError) as ei:
        lat.bodies()
    assert ei.value.code == code


def context_still_usable():
    lat = swimmer()
    lat.step(3)
    lat.sync()
    assert np.isfinite(lat.bodies()).all()


@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_nan_populations_latch_e_nan(precision):
    lat = swimmer(precision=precision)
    lat.step(2)
    pop = lat.pop()
    pop[:, :, :, :] = np.nan
    lat.set_pop(pop)
    lat.step(1)
    expect_error(lat, lbm.E_NAN)
    lat.close()
    context_still_usable()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_body_faster_than_the_step_limit_latches_e_unstable(precision):
    lat = swimmer(precision=precision)
    lat.step(2)
    s = lat.bodies()[1].copy()
    s[7:10] = (0.8, 0.0, 0.0)            # above LBM_MAX_BODY_STEP = 0.5 per step
    lat.set_body_state(1, s)
    lat.step(1)
    expect_error(lat, lbm.E_UNSTABLE)
    lat.close()
    context_still_usable()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_full_cell_list_latches_e_links(precision):
    sc = wl.Scenario("failure", 32, 32, 32, 1.0)
    wl.add_swimmer(sc, (16.3, 15.8, 16.1), (1.0, 0.0, 0.0, 0.0), (wl.SPHERE,) * 3, 3.0, 0.0,
                   9.0, 0.01, 0.005, 1e-3, 100.0, density=2.0)
    lat = lbm.Lattice(32, 32, 32, 1.0, precision=precision)
    lat.debug_set(lbm.DEBUG_CELL_LIST_CAP, 8)      # a body's shell alone lists ~10^2 cells
    for b in sc.bodies:
        lat.add_body(b.shape, b.radius, b.length, b.mass, b.pos, b.orient)
    lat.step(1)
    expect_error(lat, lbm.E_LINKS)
    lat.close()
    context_still_usable()


@pytest.mark.parametrize("precision,blocks", [("f32", 2), ("f64", 1), ("f16", 2)])
def test_expired_bulk_copy_wait_latches_e_timeout(precision, blocks):
    lat = lbm.Lattice(64, 32, 32, 1.0, precision=precision)
    lat.add_body(wl.SPHERE, 3.0, 0.0, 300.0, (20.3, 16.2, 15.8))
    lat.tune(-1, blocks)
    lat.debug_set(lbm.DEBUG_EXPIRE_WAITS, 1)
    lat.step(1)
    expect_error(lat, lbm.E_TIMEOUT)
    lat.close()
    # the same shape with the normal bound runs and reports nothing
    lat = lbm.Lattice(64, 32, 32, 1.0, precision=precision)
    lat.add_body(wl.SPHERE, 3.0, 0.0, 300.0, (20.3, 16.2, 15.8))
    lat.tune(-1, blocks)
    lat.step(2)
    lat.sync()
    assert np.isfinite(lat.pop()).all()
    lat.close()
    context_still_usable()


def test_error_surfaces_at_the_wait_of_an_asynchronous_read(cuda):
    """A read enqueued after the failing step carries the status word with
    it: lbm_wait_ticket reports the latched error."""
    lat = swimmer(precision="f32")
    lat.step(2)
    buf = cuda.empty((lat.nbodies, 13), dtype=cuda.float64, pin_memory=True).numpy()
    t = lat.bodies_async(buf)
    lat.wait(t)                                        # no error yet
    st = lat.bodies()[1].copy()
    st[7:10] = (0.8, 0.0, 0.0)                         # above LBM_MAX_BODY_STEP = 0.5 per step
    lat.set_body_state(1, st)
    lat.step(1)
    t = lat.bodies_async(buf)
    with pytest.raises(lbm.LbmError) as ei:
        lat.wait(t)
    assert ei.value.code == lbm.E_UNSTABLE
    lat.close()
    context_still_usable()

