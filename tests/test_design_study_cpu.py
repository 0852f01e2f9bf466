"""The design study's swimmers against the paper's own tables (no GPU).

Table 1 prints each design's total length and width; Tables 3, A1-A3 print
the geometric factor K of Eq. K.  The reconstructed designs (the capsule
placement and the surface-gap reading of "rest length") must reproduce the
totals exactly and K to the printed two digits, and the protocol's lattice
parameters must give the paper's tau = 2/3, omega_0 = 6 omega and the
damping ratio of the printed k, gamma, m (0.081).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1108_0786_gb300 import analysis, design_study as ds, workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def extents(b):
    """Half-extents of a body along world z and across (x)."""
    if b.shape == wl.SPHERE:
        return b.radius, b.radius
    along_z = abs(ds._rot(b.orient)[2, 0]) > 0.5
    return (b.radius + 0.5 * b.length, b.radius) if along_z else (b.radius, b.radius + 0.5 * b.length)


@pytest.mark.parametrize("label", list(ds.DESIGNS))
def test_design_reproduces_table_1_totals_and_K(label):
    sc, r_eff = ds.design(label)
    z = [b.pos[2] for b in sc.bodies]
    hz = [extents(b)[0] for b in sc.bodies]
    hx = [extents(b)[1] for b in sc.bodies]
    total = (z[2] + hz[2]) - (z[0] - hz[0])
    width = 2 * max(hx)
    want_total, want_width = GOLDEN["table1"][label][0], GOLDEN["table1"][label][1]
    assert abs(total - want_total) < 1e-9 and abs(width - want_width) < 1e-9
    K = analysis.ga_geometric_factor(*r_eff, z[1] - z[0], z[2] - z[1])
    assert abs(K - GOLDEN["ga_parameters"][label][0]) <= 0.6e-4, (label, K)
    # the drive axis of every body points along the swimming axis z
    for d in sc.drives:
        b = sc.bodies[d.body]
        np.testing.assert_allclose(ds._rot(b.orient) @ np.asarray(d.axis), [0, 0, 1], atol=1e-12)
    # bodies start clear of each other and of the walls
    assert z[1] - z[0] > hz[0] + hz[1] and z[2] - z[1] > hz[1] + hz[2]
    assert all(b.pos[0] - hx[i] > -0.5 and b.pos[0] + hx[i] < sc.nx - 0.5 for i, b in enumerate(sc.bodies))


def test_protocol_parameters_in_lattice_units():
    p = ds.lattice_parameters()
    assert abs(p["tau"] - 2.0 / 3.0) < 1e-3
    assert abs(p["mass"] - 400.0) < 1e-9
    w0 = math.sqrt(p["k"] / p["mass"])
    assert abs(w0 / p["omega"] - 6.0) < 0.03     # 6.02 from the printed k and m
    assert abs(p["gamma"] / (2 * math.sqrt(p["k"] * p["mass"])) - 0.081) < 1e-3
    assert abs(p["omega"] - GOLDEN["omega_printed"]) < 5e-6


def test_switch_off_times_and_delay():
    sc, _ = ds.design("a")
    t_offs = sorted({d.t_off for d in sc.drives})
    assert t_offs == [140580, 147609]
    assert [d.t_off for d in sc.drives if d.body == 0] == [140580]
    delayed = [d for d in sc.drives if d.phase > 0]
    assert all(abs(d.phase / (2 * math.pi * d.freq) - 7029) < 1e-9 for d in delayed)


def test_analysis_recovers_a_synthetic_cycle():
    """Bodies moving on prescribed arms recover the set amplitudes, the
    phase lag, the drift speed and the geometric factor."""
    sc, r_eff = ds.design("a")
    T = ds.PERIOD
    w = 2 * math.pi / T
    t = np.arange(4 * T, 5 * T + 1, dtype=np.float64)
    u, d1, d2, phi = 9e-6, 2.5, 3.8, 0.9
    z1 = 99.5 + u * t
    states = np.zeros((len(t), 3, 13))
    states[:, :, 3] = 1.0
    states[:, 1, 2] = z1
    states[:, 0, 2] = z1 - (16 + d1 * np.cos(w * t + phi))
    states[:, 2, 2] = z1 + (16 + d2 * np.cos(w * t))
    states[:, 1, 9] = u
    res = ds.analyse(sc, r_eff, states, 4 * T)
    assert abs(res["u_swim"] - u) < 1e-12
    assert abs(res["d1"] - d1) < 1e-9 and abs(res["d2"] - d2) < 1e-9
    assert abs(res["sin_dphi"] - math.sin(phi)) < 1e-9
    assert abs(res["K"] - 0.004557) < 2e-6
