"""Pins of the oracle's body mapping and rigid-body properties (Sec. 2.2-2.3).

A cell is an obstacle cell when its centre lies inside a body.  For a sphere
centred on a lattice point the solid cells are the integer points of a ball,
whose counts are the cubic-lattice sequence OEIS A000605 (1, 7, 19, 27, 33,
57, 81, 81, 93, 123, ... for norm <= 0, 1, 2, ...).  The capsule count is
worked out by hand in the test.  Radii are taken 1e-6 above the integer value
so that no lattice point lies within rounding of the surface.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import workloads as wl

A000605 = [1, 7, 19, 27, 33, 57, 81, 81, 93, 123, 147]


def solid_count(shape, r, l, pos, orient=(1.0, 0.0, 0.0, 0.0), n=16):
    o = oracle.Oracle(n, n, n, 1.0)
    o.add_body(shape, r, l, 1e6, pos, orient)
    o.step(1)
    return int((o.flags() > 0).sum()), o


@pytest.mark.parametrize("r2", [1, 2, 4, 9])
def test_sphere_on_lattice_point_matches_a000605(r2):
    count, _ = solid_count(wl.SPHERE, math.sqrt(r2) + 1e-6, 0.0, (8.0, 8.0, 8.0))
    assert count == A000605[r2]


def test_sphere_across_the_periodic_boundary():
    # centred on the corner lattice point: the ball wraps onto all 8 corners
    count, o = solid_count(wl.SPHERE, 3.000001, 0.0, (0.0, 0.0, 0.0))
    assert count == 123
    fl = o.flags()
    assert fl[0, 0, 0] and fl[15, 15, 15] and fl[0, 15, 0]


def test_capsule_count_by_hand():
    """Capsule r = 2, l = 4 along x at a lattice point.

    |x| <= 2: the 13 points of the disc y^2 + z^2 <= 4 (5 planes);
    |x| = 3: (|x| - 2)^2 + y^2 + z^2 <= 4 -> y^2 + z^2 <= 3: 9 points (2 planes);
    |x| = 4: only the axis point (2 planes).  Total 5*13 + 2*9 + 2*1 = 85.
    """
    count, _ = solid_count(wl.CAPSULE, 2.000001, 4.0, (8.0, 8.0, 8.0))
    assert count == 85
    # the same capsule turned by 90 degrees about z lies along y
    c = math.cos(math.pi / 4)
    count_y, o = solid_count(wl.CAPSULE, 2.000001, 4.0, (8.0, 8.0, 8.0), (c, 0.0, 0.0, c))
    assert count_y == 85
    fl = o.flags()
    assert fl[8, 12, 8] and not fl[8, 8, 12]


def test_solid_volume_approaches_body_volume():
    count, _ = solid_count(wl.SPHERE, 8.0, 0.0, (16.3, 15.8, 16.1), n=34)
    assert abs(count / (4.0 / 3.0 * math.pi * 8 ** 3) - 1.0) < 0.02
    count, _ = solid_count(wl.CAPSULE, 5.0, 10.0, (16.3, 15.8, 16.1), (0.9, 0.2, 0.3, 0.1), n=34)
    assert abs(count / (math.pi * 25 * 10 + 4.0 / 3.0 * math.pi * 125) - 1.0) < 0.03


def voxel_inertia(r, l, h=0.02):
    """Numerical principal moments per unit mass of a solid capsule along x."""
    xs = np.arange(-(l / 2 + r) + h / 2, l / 2 + r, h)
    ys = np.arange(-r + h / 2, r, h)
    X, Y, Z = np.meshgrid(xs, ys, ys, indexing="ij")
    s = np.clip(X, -l / 2, l / 2)
    inside = (X - s) ** 2 + Y ** 2 + Z ** 2 <= r * r
    n = inside.sum()
    ixx = ((Y ** 2 + Z ** 2) * inside).sum() / n
    iyy = ((X ** 2 + Z ** 2) * inside).sum() / n
    vol = n * h ** 3
    return vol, ixx, iyy


@pytest.mark.parametrize("r,l", [(1.0, 0.0), (1.0, 2.0), (1.0, 0.5)])
def test_inertia_against_voxel_integration(r, l):
    shape = wl.SPHERE if l == 0 else wl.CAPSULE
    o = oracle.Oracle(4, 4, 4, 1.0)
    m = 3.7
    o.add_body(shape, r, l, m, (2.0, 2.0, 2.0))
    vol, i1, i2, i3 = o.body_props(0)
    v_num, ixx, iyy = voxel_inertia(r, l)
    assert abs(vol / v_num - 1.0) < 5e-3
    assert abs(i1 / (m * ixx) - 1.0) < 5e-3
    assert abs(i2 / (m * iyy) - 1.0) < 5e-3
    assert i2 == i3


def test_overlapping_bodies_are_an_error():
    o = oracle.Oracle(16, 16, 16, 1.0)
    o.add_body(wl.SPHERE, 3.0, 0.0, 100.0, (6.0, 8.0, 8.0))
    o.add_body(wl.SPHERE, 3.0, 0.0, 100.0, (10.5, 8.0, 8.0))
    with pytest.raises(oracle.OracleError) as ei:
        o.step(1)
    assert ei.value.code == oracle.E_OVERLAP


def test_body_crossing_a_wall_is_an_error():
    o = oracle.Oracle(16, 16, 16, 1.0, bc=wl.PERIODIC_X)
    o.add_body(wl.SPHERE, 3.0, 0.0, 100.0, (8.0, 2.0, 8.0))
    with pytest.raises(oracle.OracleError) as ei:
        o.step(1)
    assert ei.value.code == oracle.E_OUTSIDE
