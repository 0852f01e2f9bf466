"""Three-sphere swimmer set-up and Golestanian-Ajdari analysis (Sec. 5.3).

A swimmer of three spheres along x is driven with the protocol of Sec. 3.3.
The drive is set to a quasi-static regime like the paper's (spring
frequency omega_0 = 6 omega, damping ratio 0.07, body Reynolds number
~0.06), the arm lengths are fitted over the last full period with Eq. arms,
and the measured speed of the middle body over that period is compared with
u_GA = K d1 d2 omega sin(phi1 - phi2) (Eq. V_GA, Eq. K).
"""
import math

import numpy as np

from paper_1108_0786_gb300 import analysis, workloads as wl


def swimmer_scenario(nx, ny, nz, r, arm, T, deflection, tau=1.0, density=2.0):
    sc = wl.Scenario("GA swimmer", nx, ny, nz, tau)
    m = density * wl.sphere_volume(r)
    omega = 2 * math.pi / T
    k = m * (6.0 * omega) ** 2
    gamma = 2 * 0.07 * math.sqrt(m * k)
    wl.add_swimmer(sc, (nx / 2 + 0.3, ny / 2 + 0.2, nz / 2 - 0.1), (1.0, 0.0, 0.0, 0.0),
                   (wl.SPHERE,) * 3, r, 0.0, arm, k, gamma, deflection * k, T)
    return sc


def ga_analysis(x, r, T):
    """x: body x positions over the last period, shape (T + 1, 3) for (B2, B1, B3)."""
    omega = 2 * math.pi / T
    t = np.arange(len(x))
    lb1, d1, p1 = analysis.fit_arm(t, x[:, 1] - x[:, 0], omega)
    lb2, d2, p2 = analysis.fit_arm(t, x[:, 2] - x[:, 1], omega)
    K = analysis.ga_geometric_factor(r, r, r, lb1, lb2)
    u_ga = analysis.ga_velocity(K, d1, d2, omega, math.sin(p1 - p2))
    u_swim = (x[-1, 1] - x[0, 1]) / T
    return {"d1": d1, "d2": d2, "u_ga": u_ga, "u_swim": u_swim, "ratio": u_swim / u_ga}


def oracle_last_period(o, T, periods):
    """Advance an oracle swimmer and record x over its last period."""
    o.step(int((periods - 1) * T))
    xs = [o.bodies()[:, 0].copy()]
    for _ in range(T):
        o.step(1)
        xs.append(o.bodies()[:, 0].copy())
    return np.array(xs)
