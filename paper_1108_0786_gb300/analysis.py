"""Trajectory analysis of three-body swimmers (Sec. 5.2-5.3 of the paper).

Post-processing utilities, not part of the time step: the Golestanian-Ajdari
prediction of the swimming speed (Eq. V_GA, Eq. K), the fit of the arm
lengths to Eq. arms, the swimming speed over the last full cycle, the
Reynolds numbers of Eq. Re / ReSwimmer / ReBody, Lighthill's efficiency
(Eq. eff) and the conversion of the paper's physical parameters to lattice
units.  All inputs and outputs are plain numbers or numpy arrays.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np


def ga_geometric_factor(r1: float, r2: float, r3: float, l1: float, l2: float) -> float:
    """K of Eq. K: 3 r1 r2 r3 / (2 (r1+r2+r3)^2) [1/l1^2 + 1/l2^2 - 1/(l1+l2)^2]."""
    s = r1 + r2 + r3
    return 3.0 * r1 * r2 * r3 / (2.0 * s * s) * (1.0 / l1 ** 2 + 1.0 / l2 ** 2 - 1.0 / (l1 + l2) ** 2)


def ga_velocity(K: float, d1: float, d2: float, omega: float, sin_dphi: float) -> float:
    """u_GA = K d1 d2 omega sin(phi1 - phi2) (Eq. V_GA)."""
    return K * d1 * d2 * omega * sin_dphi


def fit_arm(t: Sequence[float], length: Sequence[float], omega: float) -> Tuple[float, float, float]:
    """Least-squares fit of l(t) = l_bar + d cos(omega t + phi) (Eq. arms).

    Returns (l_bar, d, phi) with d >= 0 and phi in (-pi, pi].
    """
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(length, dtype=np.float64)
    B = np.column_stack([np.ones_like(t), np.cos(omega * t), np.sin(omega * t)])
    (lb, c, s), *_ = np.linalg.lstsq(B, y, rcond=None)
    # d cos(wt + phi) = d cos(phi) cos(wt) - d sin(phi) sin(wt)
    d = math.hypot(c, s)
    phi = math.atan2(-s, c)
    return float(lb), float(d), float(phi)


def swimming_speed(x_centre: Sequence[float], period: int) -> float:
    """u_swim = Delta / T from the central body's last full cycle (Sec. 5.2)."""
    x = np.asarray(x_centre, dtype=np.float64)
    return float((x[-1] - x[-1 - int(period)]) / period)


def reynolds(u: float, length: float, nu: float) -> float:
    """Re = u l / nu (Eq. Re)."""
    return u * length / nu


def lighthill_efficiency(mu: float, r_eff: float, u_swim: float, period: int,
                         drive_forces: np.ndarray, velocities: np.ndarray) -> float:
    """Eq. eff: 6 pi mu r_eff u^2 / ((1/T) sum_t sum_i F_dri,i(t) . u_i(t)).

    ``drive_forces`` and ``velocities`` have shape (steps, bodies, 3) over the
    last full cycle (one sample per time step, dt = 1).
    """
    power = np.einsum("tbi,tbi->", np.asarray(drive_forces), np.asarray(velocities)) / period
    return 6.0 * math.pi * mu * r_eff * u_swim ** 2 / power


def lattice_units(dx: float, period_steps: int, omega_si: float, mass_unit: float) -> dict:
    """Conversion factors from SI to lattice units (dx = dt = 1).

    dt follows from the period: omega_lattice = 2 pi / T = omega_si dt.
    """
    dt = (2.0 * math.pi / period_steps) / omega_si
    return {"dx": dx, "dt": dt, "mass": mass_unit,
            "viscosity": dt / dx ** 2,            # nu_L = nu dt / dx^2
            "force": dt ** 2 / (mass_unit * dx),  # F_L = F dt^2 / (M dx)
            "stiffness": dt ** 2 / mass_unit,     # k_L = k dt^2 / M
            "damping": dt / mass_unit}            # gamma_L = gamma dt / M


def tau_from_viscosity(nu_lattice: float) -> float:
    """LBGK relaxation time for a lattice viscosity: nu = (tau - 1/2) / 3."""
    return 3.0 * nu_lattice + 0.5
