"""Exact invariants of the oracle's coupled step.

Each test states an identity that follows from the method itself (Sec. 2.1 and
2.3) and holds to round-off at any size: the rest state is a fixed point, BGK
with bounce-back at resting walls conserves mass, a periodic box conserves
momentum, Guo's forcing adds exactly g per cell and step, the momentum-exchange
force equals the momentum the stream exchanges, and fluid plus bodies conserve
momentum when the net drive is zero.
"""
import numpy as np
import pytest

import oracle
from oracle_helpers import momentum
from paper_1108_0786_gb300 import workloads as wl

E, W = oracle.lattice()


def random_pop(shape, seed, amp=1e-3):
    rng = wl.SplitMix64(seed)
    nz, ny, nx = shape
    n = 19 * nx * ny * nz
    noise = np.array([rng.uniform(-amp, amp) for _ in range(n)]).reshape(19, nz, ny, nx)
    return W[:, None, None, None] * (1.0 + noise)


def test_rest_state_is_a_fixed_point_with_resting_bodies():
    # bodies about 3.5 times denser than the fluid: explicit momentum-exchange
    # coupling amplifies round-off for bodies much lighter than the fluid
    o = oracle.Oracle(20, 18, 16, 0.8)
    o.add_body(wl.SPHERE, 3.0, 0.0, 400.0, (6.3, 9.1, 7.7))
    o.add_body(wl.CAPSULE, 2.5, 4.0, 500.0, (14.2, 8.4, 8.6), (0.9, 0.1, 0.3, 0.2))
    o.step(30)
    pop = o.pop()
    flags = o.flags()
    fluid = flags == 0
    assert fluid.sum() < fluid.size
    assert np.abs(pop[:, fluid] - W[:, None]).max() < 1e-15
    # link terms are O(0.1) each and cancel in pairs: round-off only
    assert np.abs(o.forces()).max() < 1e-13
    b = o.bodies()
    assert np.abs(b[:, 7:]).max() < 1e-15


def test_mass_conserved_with_walls_and_resting_obstacle():
    # walls in y, periodic x and z, a resting (very heavy) sphere
    o = oracle.Oracle(14, 12, 10, 0.7, bc=wl.PERIODIC_X | 4)
    o.add_body(wl.SPHERE, 2.6, 0.0, 1e30, (6.4, 5.2, 4.9))
    o.set_pop(random_pop(o.shape, 7))
    o.step(1)
    fluid = o.flags() == 0
    m0 = o.pop()[:, fluid].sum()
    for _ in range(40):
        o.step(1)
        assert abs(o.pop()[:, fluid].sum() - m0) < 1e-12 * m0
    assert np.array_equal(o.flags() == 0, fluid)


def test_momentum_conserved_in_periodic_box():
    o = oracle.Oracle(9, 8, 7, 0.9)
    o.set_pop(random_pop(o.shape, 11))
    p0 = momentum(random_pop(o.shape, 11), E)
    o.step(1)
    p1 = momentum(o.pop(), E)
    assert np.allclose(p1, p0, atol=1e-13, rtol=0)
    for _ in range(20):
        o.step(1)
        assert np.allclose(momentum(o.pop(), E), p0, atol=1e-13, rtol=0)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_guo_forcing_adds_g_per_cell_and_step(tau):
    g = np.array([2e-5, -1e-5, 3e-6])
    o = oracle.Oracle(8, 6, 5, tau, g=g)
    o.set_pop(random_pop(o.shape, 5))
    o.step(1)
    prev = momentum(o.pop(), E)
    for _ in range(10):
        o.step(1)
        cur = momentum(o.pop(), E)
        assert np.allclose(cur - prev, g * o.cells, atol=1e-13, rtol=0)
        prev = cur


def test_momentum_exchange_force_is_the_exchanged_momentum():
    """P_fluid(n+1) = P_fluid(n) - F_hydro(n) while no cell changes its flag.

    A heavy sphere moves through fluid at rest with a prescribed velocity and
    rotation; the fluid loses exactly the momentum the body receives.
    """
    o = oracle.Oracle(24, 22, 20, 0.8)
    b = o.add_body(wl.SPHERE, 4.0, 0.0, 1e30, (11.3, 10.6, 9.8))
    o.set_body_state(b, [11.3, 10.6, 9.8, 1, 0, 0, 0, 2e-3, -1e-3, 5e-4, 1e-4, 3e-4, -2e-4])
    o.step(1)
    checked = 0
    for _ in range(60):
        p0, f0, fl0 = momentum(o.pop(), E), o.forces()[0, :3], o.flags()
        o.step(1)
        if not np.array_equal(o.flags(), fl0):
            continue
        p1 = momentum(o.pop(), E)
        # |F| ~ 0.1; the bound is the round-off of summing ~2e5 populations
        assert np.allclose(p1 - p0, -f0, atol=1e-12, rtol=0)
        checked += 1
    assert checked > 40


def test_swimmer_conserves_fluid_plus_body_momentum():
    """With zero net drive and central springs, P_fluid + sum m V is constant
    between remap events (Eq. FB1 makes the drive sum vanish, Sec. 3.3).

    The swimmer lies on the lattice planes y = z = 16, so no body turns and
    the three drive axes stay parallel (the drive acts along each body's own
    x axis)."""
    sc = wl.Scenario("swimmer", 32, 32, 32, 1.0)
    wl.add_swimmer(sc, (16.2, 16.0, 16.0), (1.0, 0.0, 0.0, 0.0), (wl.SPHERE,) * 3, 3.0, 0.0,
                   10.0, 0.01, 0.005, 5e-3, 50.0)
    o = oracle.from_scenario(sc)
    m = np.array([b.mass for b in sc.bodies])
    v_prev = o.bodies()[:, 7:10]
    o.step(1)
    checked = 0
    q_ref = momentum(o.pop(), E) + (m[:, None] * v_prev).sum(axis=0)
    for _ in range(150):
        fl0 = o.flags()
        v_prev = o.bodies()[:, 7:10]
        o.step(1)
        q = momentum(o.pop(), E) + (m[:, None] * v_prev).sum(axis=0)
        if not np.array_equal(o.flags(), fl0):
            q_ref = q
            continue
        assert np.allclose(q, q_ref, atol=1e-12, rtol=0)
        checked += 1
    assert checked > 100
    assert np.abs(o.bodies()[:, 7:10]).max() > 1e-5      # the bodies did move


def test_mirror_symmetric_setup_has_no_transverse_force_or_torque():
    """A sphere centred on lattice planes y = 8 and z = 8 moving along x."""
    o = oracle.Oracle(24, 17, 17, 1.0)
    b = o.add_body(wl.SPHERE, 3.5, 0.0, 1e30, (10.37, 8.0, 8.0))
    o.set_body_state(b, [10.37, 8, 8, 1, 0, 0, 0, 1e-3, 0, 0, 0, 0, 0])
    for _ in range(25):
        o.step(1)
        f = o.forces()[0]
        assert abs(f[0]) > 1e-8
        assert np.abs(f[1:]).max() < 1e-13      # round-off of ~600 link terms
