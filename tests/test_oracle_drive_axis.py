"""Drive terms along a body-frame axis (the paper's perpendicular capsules,
Sec. 5.1, are driven along the swimming direction, not along their own axis).

Pins: (1) the world-frame drive direction is R(q) a: bodies turned by q and
driven along a = R(q)^T e move exactly like unturned bodies driven along e
(a transposed rotation would send them elsewhere); (2) the reverse mode's
drive and orientation gradients with non-default axes against central
differences, with and without fluid.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from adjoint_helpers import axis_swimmer as swimmer


@pytest.mark.parametrize("fluid", [False, True])
def test_turned_bodies_driven_along_the_mapped_axis_move_alike(fluid):
    opts = 0 if fluid else oracle.OPT_NO_FLUID
    q = (0.8, 0.3, -0.4, 0.33)
    ref = oracle.from_scenario(swimmer((1, 0, 0, 0), (1, 0, 0)), opts)
    turned = oracle.from_scenario(swimmer(q, (1, 0, 0)), opts)
    ref.step(80)
    turned.step(80)
    # spheres: the turn changes neither the map nor the hydrodynamics
    np.testing.assert_allclose(turned.bodies()[:, 0:3], ref.bodies()[:, 0:3], rtol=0, atol=1e-11)
    np.testing.assert_allclose(turned.bodies()[:, 7:10], ref.bodies()[:, 7:10], rtol=0, atol=1e-13)
    # the same axis without the turn drives along another world direction
    wrong = oracle.from_scenario(dataclasses.replace(swimmer(q, (1, 0, 0)), bodies=swimmer(
        (1, 0, 0, 0), (1, 0, 0)).bodies), opts)
    wrong.step(80)
    assert np.abs(wrong.bodies()[:, 0:3] - ref.bodies()[:, 0:3]).max() > 1e-3


@pytest.mark.parametrize("fluid", [False, True])
def test_reverse_mode_with_drive_axes(fluid):
    opts = 0 if fluid else oracle.OPT_NO_FLUID
    q = (0.8, 0.3, -0.4, 0.33)
    seed = np.zeros((3, 13))
    seed[1, 0] = 1.0
    seed[0, 2] = 0.5
    n = 50
    g = oracle.from_scenario(swimmer(q, (1, 0, 0)), opts).adjoint(n, seed)

    def J(sc=None, dstate=None):
        o = oracle.from_scenario(sc or swimmer(q, (1, 0, 0)), opts)
        if dstate is not None:
            st = o.bodies() + dstate
            for b in range(3):
                o.set_body_state(b, st[b])
        o.step(n)
        return float((o.bodies() * seed).sum()), o.flag_digest
    for term in (0, 2, 3):
        h = 1e-7
        sp = swimmer(q, (1, 0, 0))
        sm = swimmer(q, (1, 0, 0))
        sp.drives[term] = dataclasses.replace(sp.drives[term], amp=sp.drives[term].amp + h)
        sm.drives[term] = dataclasses.replace(sm.drives[term], amp=sm.drives[term].amp - h)
        (jp, dp), (jm, dm) = J(sp), J(sm)
        assert dp == dm
        fd = (jp - jm) / (2 * h)
        tol = 1e-6 * abs(fd) + 100 * 2.2e-16 * max(abs(jp), abs(jm)) / h
        assert abs(g["drive"][term, 0] - fd) <= tol, (term, g["drive"][term, 0], fd)
    # orientation of body 0 (the drive direction turns with it; spheres keep
    # the map): quaternion components through R(q) a
    for comp in (3, 4, 6):
        h = 1e-5
        d = np.zeros((3, 13))
        d[0, comp] = h
        (jp, dp), (jm, dm) = J(dstate=d), J(dstate=-d)
        assert dp == dm
        fd = (jp - jm) / (2 * h)
        # set_body_state renormalises q: compare with the gradient projected
        # on the tangent of the unit sphere
        q0 = np.asarray(q) / np.linalg.norm(q)
        gq = g["state"][0, 3:7]
        tang = gq - q0 * (q0 @ gq)
        e = np.zeros(4)
        e[comp - 3] = 1.0
        tol = 1e-5 * abs(fd) + 100 * 2.2e-16 * max(abs(jp), abs(jm)) / h
        assert abs(tang @ e - fd) <= tol, (comp, tang @ e, fd)
