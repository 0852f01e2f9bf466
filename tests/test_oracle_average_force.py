"""The averaged-load option (not in the paper: the rigid-body step takes the
mean hydrodynamic force and torque of steps n and n-1, a stabiliser of the
explicit coupling for bodies near or below the fluid's density).

Pin: the fluid still gives up F^n at each stream while the bodies take the
mean of F^n and F^(n-1), so P_fluid + sum m V + F^(n-1) / 2 is conserved
between remap events (the plain coupling conserves P_fluid + sum m V; the
identity telescopes).  A wrong weight or a wrong lag breaks it.  Also: the
first step is not averaged, and the reverse mode refuses the option.
"""
import numpy as np
import pytest

import oracle
from oracle_helpers import momentum
from paper_1108_0786_gb300 import workloads as wl

E, W = oracle.lattice()


def swimmer():
    sc = wl.Scenario("swimmer", 32, 32, 32, 1.0)
    wl.add_swimmer(sc, (16.2, 16.0, 16.0), (1.0, 0.0, 0.0, 0.0), (wl.SPHERE,) * 3, 3.0, 0.0,
                   10.0, 0.01, 0.005, 5e-3, 50.0)
    return sc


def test_fluid_plus_body_momentum_with_the_half_lagged_load():
    sc = swimmer()
    o = oracle.from_scenario(sc, oracle.OPT_AVERAGE_FORCE)
    m = np.array([b.mass for b in sc.bodies])
    o.step(2)
    ref = None
    checked = 0
    for _ in range(150):
        fl0 = o.flags()
        v_prev = o.bodies()[:, 7:10]
        f_prev = o.forces()[:, 0:3].sum(axis=0)      # F^(n-1): the load the coming stream exchanges
        o.step(1)
        q = momentum(o.pop(), E) + (m[:, None] * v_prev).sum(axis=0) + 0.5 * f_prev
        if not np.array_equal(o.flags(), fl0) or ref is None:
            ref = q
            continue
        assert np.allclose(q, ref, atol=1e-12, rtol=0)
        checked += 1
    assert checked > 100
    assert np.abs(o.bodies()[:, 7:10]).max() > 1e-5


def test_first_step_is_not_averaged_and_later_steps_differ():
    sc = swimmer()
    plain, avg = oracle.from_scenario(sc), oracle.from_scenario(sc, oracle.OPT_AVERAGE_FORCE)
    plain.step(1)
    avg.step(1)
    assert np.array_equal(plain.bodies(), avg.bodies())
    plain.step(5)
    avg.step(5)
    assert np.abs(plain.bodies()[:, 7:10] - avg.bodies()[:, 7:10]).max() > 1e-9


def test_reverse_mode_refuses_the_averaged_load():
    o = oracle.from_scenario(swimmer(), oracle.OPT_AVERAGE_FORCE)
    with pytest.raises(oracle.OracleError):
        o.adjoint(3, np.zeros((3, 13)))
