"""The swimmer analysis against the numbers the paper prints (Sec. 5.2-5.3).

Fixture ``golden/paper_tables.json`` holds Tables 1-6 and A1-A3 as printed.
The printed inputs carry two to three significant digits, which bounds how
well recomputed values can agree.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1108_0786_gb300 import analysis

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "paper_tables.json")) as fh:
    TABLES = json.load(fh)

OMEGA = 2 * math.pi / TABLES["period_steps"]


def test_printed_omega_is_the_period():
    assert abs(OMEGA - TABLES["omega_printed"]) < 0.05 * TABLES["omega_printed"]


@pytest.mark.parametrize("design", sorted(TABLES["ga_parameters"]))
def test_ga_velocity_from_printed_parameters(design):
    """Eq. V_GA with the printed K, d1, d2 and sin reproduces the printed u_GA."""
    K, d1, d2, s = TABLES["ga_parameters"][design]
    u_ga = analysis.ga_velocity(K, d1, d2, OMEGA, s)
    printed = TABLES["velocities"][design][1] * 1e-6
    assert abs(u_ga / printed - 1.0) < 0.05


@pytest.mark.parametrize("design", sorted(TABLES["velocities"]))
def test_printed_error_bounds(design):
    """Error = |u_GA - u_swim| / u_GA * 100 stays below the printed bound."""
    u_swim, u_ga, bound, _ = TABLES["velocities"][design]
    err = abs(u_ga - u_swim) / u_ga * 100
    assert err < bound + 0.5


def test_geometric_factor_of_the_sphere_swimmers():
    """Eq. K with the Table 1 geometry: design (a) spheres r = 4 with arms of
    16 (8-cell gap plus two radii); design (q) spheres r = 8 with arms of 24."""
    K_a = analysis.ga_geometric_factor(4, 4, 4, 16, 16)
    K_q = analysis.ga_geometric_factor(8, 8, 8, 24, 24)
    assert abs(K_a - 0.0045) < 1e-4
    assert abs(K_q - 0.0040) < 1e-4
    # the total length of Table 1 is two arms plus two radii
    assert TABLES["table1"]["a"][0] == 16 + 16 + 2 * 4
    assert TABLES["table1"]["q"][0] == 24 + 24 + 2 * 8


@pytest.mark.parametrize("design", sorted(TABLES["table1"]))
def test_swimmer_reynolds_numbers_fix_the_lattice_viscosity(design):
    """Eq. ReSwimmer with the printed u_swim and rest length reproduces the
    printed Re_swim for nu = 1/18 in lattice units, i.e. tau = 2/3: the value
    the paper's physical parameters give (nu = 7.36e-5 m^2/s, dx = 1e-6 m,
    T = 28116 steps at omega = 296057.86703 1/s)."""
    length, _, re_printed = TABLES["table1"][design]
    u_swim = TABLES["velocities"][design][0] * 1e-6
    nu = 1.0 / 18.0
    assert abs(analysis.reynolds(u_swim, length, nu) / (re_printed * 1e-3) - 1.0) < 0.01
    units = analysis.lattice_units(1e-6, TABLES["period_steps"], 296057.86703, 1.36e-15)
    nu_l = 7.36e-5 * units["viscosity"]
    assert abs(nu_l - nu) < 1e-4
    assert abs(analysis.tau_from_viscosity(nu_l) - 2.0 / 3.0) < 1e-3


def test_fit_arm_recovers_amplitude_and_phase():
    t = np.arange(400)
    w = 2 * math.pi / 400
    lb, d, phi = analysis.fit_arm(t, 16.0 + 2.5 * np.cos(w * t + 0.7), w)
    assert abs(lb - 16.0) < 1e-12 and abs(d - 2.5) < 1e-12 and abs(phi - 0.7) < 1e-12
