"""Closed-form flows that pin the oracle's fluid solver (Sec. 2.1, 2.3).

- plane Poiseuille flow between halfway bounce-back walls (Eq. 4) with Guo's
  body force: BGK gives the exact parabola plus a uniform slip
  u_s = (2 g / 3 nu) ((tau - 1/2)^2 - 3/16), which vanishes at
  (tau - 1/2)^2 = 3/16 (He, Zou, Luo & Dembo 1997; Ginzburg's Lambda = 3/16);
- square-duct flow against its Fourier series;
- decay of a shear wave at rate nu k^2 with nu = (tau - 1/2) / 3;
- drag on a fixed sphere in a periodic array against Stokes' law with the
  Hasimoto / Sangani-Acrivos correction, and the force balance F = g N_fluid;
- torque on a rotating sphere against the rotlet law T = -8 pi mu r^3 Omega
  (this exercises the moving-wall correction of the bounce-back rule).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import workloads as wl

TAU_STAR = 0.5 + math.sqrt(3.0) / 4.0


def poiseuille(tau, H, g, steps):
    o = oracle.Oracle(1, H, 1, tau, bc=wl.PERIODIC_X | 4, g=(g, 0.0, 0.0))
    o.step(steps)
    return o.u()[0, 0, :, 0]


def test_poiseuille_exact_at_magic_tau():
    H, g = 16, 1e-6
    nu = (TAU_STAR - 0.5) / 3.0
    u = poiseuille(TAU_STAR, H, g, 6000)
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.abs(u - exact).max() < 1e-10 * exact.max()


@pytest.mark.parametrize("tau,H,steps", [(0.6, 16, 40000), (0.8, 12, 6000), (1.0, 16, 3000),
                                         (1.5, 16, 3000)])
def test_poiseuille_parabola_plus_bgk_slip(tau, H, steps):
    g = 1e-6
    nu = (tau - 0.5) / 3.0
    u = poiseuille(tau, H, g, steps)
    y = np.arange(H)
    slip = 2.0 * g / (3.0 * nu) * ((tau - 0.5) ** 2 - 3.0 / 16.0)
    exact = g / (2 * nu) * (y + 0.5) * (H - y - 0.5) + slip
    assert np.abs(u - exact).max() < 1e-7 * exact.max()


def test_poiseuille_tau1_within_one_percent_at_H32():
    H, g, tau = 32, 1e-6, 1.0
    nu = (tau - 0.5) / 3.0
    u = poiseuille(tau, H, g, 12000)
    y = np.arange(H)
    exact = g / (2 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.linalg.norm(u - exact) / np.linalg.norm(exact) < 1e-2


def duct_series(a, y, z, g, nu, nmax=199):
    """Fully developed flow in a square duct of side a; y, z from the centre."""
    s = np.zeros_like(y)
    for n in range(1, nmax + 1, 2):
        s += ((-1) ** ((n - 1) // 2) / n ** 3 *
              (1 - np.cosh(n * np.pi * z / a) / np.cosh(n * np.pi / 2)) * np.cos(n * np.pi * y / a))
    return 4 * g * a * a / (nu * np.pi ** 3) * s


@pytest.mark.parametrize("tau,steps", [(TAU_STAR, 6000), (1.0, 4000)])
def test_square_duct_against_fourier_series(tau, steps):
    a, g = 24, 1e-6
    nu = (tau - 0.5) / 3.0
    o = oracle.Oracle(1, a, a, tau, bc=wl.PERIODIC_X, g=(g, 0.0, 0.0))
    o.step(steps)
    u = o.u()[0, :, :, 0]
    c = np.arange(a) - (a - 1) / 2.0
    Z, Y = np.meshgrid(c, c, indexing="ij")
    exact = duct_series(a, Y, Z, g, nu)
    assert np.linalg.norm(u - exact) / np.linalg.norm(exact) < 2e-3


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.6])
def test_shear_wave_decays_at_nu_k2(tau):
    # the BGK decay rate carries an O(k^2) relative correction: keep k small
    L, u0 = 128, 1e-4
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / L
    o = oracle.Oracle(1, L, 1, tau)
    y = np.arange(L)
    ux = u0 * np.sin(k * y)
    pop = np.stack([oracle.equilibrium(1.0, [ux[j], 0.0, 0.0]) for j in range(L)], axis=1)
    o.set_pop(pop[:, None, :, None])
    o.step(100)

    def amplitude():
        return 2 * np.mean(o.u()[0, 0, :, 0] * np.sin(k * y))

    a1 = amplitude()
    o.step(1000)
    a2 = amplitude()
    rate = -math.log(a2 / a1) / 1000
    assert abs(rate / (nu * k * k) - 1.0) < 2e-3


def hasimoto_K(phi):
    """1/K of Sangani & Acrivos (1982) for a simple cubic array of spheres."""
    return (1 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2 + 3.9799 * phi ** (8 / 3)
            - 3.0734 * phi ** (10 / 3))


def aitken(s):
    d1, d2 = s[-1] - s[-2], s[-2] - s[-3]
    return s[-1] - d1 * d1 / (d1 - d2)


@pytest.mark.parametrize("r", [4.5, 6.0])
def test_fixed_sphere_drag_matches_stokes_hasimoto(r):
    """F = 6 pi mu r U / K(phi), U the velocity averaged over the whole cell.

    The approach to the steady state is a single slow exponential, so the
    last three samples are extrapolated with Aitken's delta-squared."""
    L, tau, g = 32, 1.0, 1e-6
    nu = (tau - 0.5) / 3.0
    o = oracle.Oracle(L, L, L, tau, g=(g, 0.0, 0.0))
    X = (L / 2 - 0.3, L / 2 + 0.2, L / 2 + 0.1)
    o.add_body(wl.SPHERE, r, 0.0, 1e30, X)
    phi = 4.0 / 3.0 * math.pi * r ** 3 / L ** 3
    u_start = g * L ** 3 * (1 - phi) * hasimoto_K(phi) / (6 * math.pi * nu * r)
    pop = oracle.equilibrium(1.0, [u_start, 0.0, 0.0])[:, None, None, None] * np.ones((1, L, L, L))
    o.set_pop(pop)
    U, F = [], []
    for _ in range(6):
        o.step(300)
        U.append(o.u()[0].sum() / L ** 3)
        F.append(o.forces()[0, 0])
    n_fluid = (o.flags() == 0).sum()
    F_inf, U_inf = aitken(F), aitken(U)
    # steady state: the drag balances the body force on all fluid cells
    assert abs(F_inf / (g * n_fluid) - 1.0) < 1e-3
    stokes = 6 * math.pi * nu * r * U_inf / hasimoto_K(phi)
    assert abs(F_inf / stokes - 1.0) < 0.05
    assert np.abs(o.forces()[0, 1:3]).max() < 0.05 * F_inf


@pytest.mark.parametrize("r", [4.5, 6.0])
def test_rotating_sphere_torque_matches_rotlet(r):
    L, tau, Om = 32, 1.0, 1e-4
    nu = (tau - 0.5) / 3.0
    o = oracle.Oracle(L, L, L, tau)
    X = (L / 2 - 0.3, L / 2 + 0.2, L / 2 + 0.1)
    o.add_body(wl.SPHERE, r, 0.0, 1e30, X)
    o.set_body_state(0, list(X) + [1, 0, 0, 0, 0, 0, 0, 0, 0, Om])
    o.step(900)
    T = o.forces()[0]
    rotlet = -8 * math.pi * nu * r ** 3 * Om
    # the torque opposes the rotation; periodic images and the staircase
    # surface change it by a few per cent
    assert 0.95 < T[5] / rotlet < 1.08
    assert np.abs(T[3:5]).max() < 0.02 * abs(T[5])
    assert np.abs(T[:3]).max() < 0.02 * abs(T[5]) / r
