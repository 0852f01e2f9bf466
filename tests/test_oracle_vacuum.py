"""The three-sphere swimmer in vacuum (Sec. 4, Fig. 9-10 of the paper).

Without fluid the swimmer is a linear system: three masses m, two damped
springs (Eq. osci_b1-b3) and the drive of Eq. FB1-FB3.  Two closed forms pin
the oracle's rigid-body part:

(i) the exact solution of the discrete recurrence the integrator defines
    (semi-implicit Euler, dt = 1): with deformations q1 = x2 - x1 + l0,
    q2 = x3 - x1 - l0 and their rates w = (w1, w2) one step is
        w' = w + Kc (-k q - gamma w + D) / m,   q' = q + w',
    with Kc = [[2, 1], [1, 2]] and D = (D2, D3) the outer drives;
    it is summed in closed form over the eigenvalues of the 4x4 step matrix
    (geometric series of the sinusoidal drive), and the centre of mass stays
    at rest because the net drive vanishes;
(ii) the steady state of the continuous equations of motion (the paper's
    Lagrangian with damping), whose amplitude has maxima at omega_0 = omega
    and omega_0 = omega / sqrt(3) (Fig. 10).

The parameters of (i) are the paper's Fig. 9 values converted to lattice
units (dx = 1e-6 m, T = 28116 steps, mass unit 1.36e-15 kg).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import workloads as wl

# Fig. 9 caption, SI units
M_SI, K_SI, GAMMA_SI, OMEGA_SI, A_SI = 5.44e-13, 1.72965, 1.57237e-7, 296057.86703, 1.0e-5
DX, T_STEPS, MASS_UNIT = 1e-6, 28116, 1.36e-15
DT = (2 * math.pi / T_STEPS) / OMEGA_SI


def lattice_params():
    m = M_SI / MASS_UNIT
    k = K_SI * DT ** 2 / MASS_UNIT
    gamma = GAMMA_SI * DT / MASS_UNIT
    a = A_SI * DT ** 2 / (MASS_UNIT * DX)
    return m, k, gamma, a


def vacuum_swimmer(m, k, gamma, a, T, x=(25.0, 50.0, 75.0), t1=math.inf, t2=math.inf):
    """Bodies B2, B1, B3 at x along the x axis; springs of rest length l0."""
    o = oracle.Oracle(1, 1, 1, 1.0, options=oracle.OPT_NO_FLUID)
    x2, x1, x3 = x
    b2 = o.add_body(wl.SPHERE, 4.0, 0.0, m, (x2, 0, 0))
    b1 = o.add_body(wl.SPHERE, 4.0, 0.0, m, (x1, 0, 0))
    b3 = o.add_body(wl.SPHERE, 4.0, 0.0, m, (x3, 0, 0))
    l0 = x1 - x2
    o.add_spring(b2, b1, k, l0, gamma)
    o.add_spring(b3, b1, k, x3 - x1, gamma)
    f = 1.0 / T
    for body, amp, phase, off in ((b2, -a, 0.0, t1), (b1, a, 0.0, t1),
                                  (b3, a, math.pi / 2, t2), (b1, -a, math.pi / 2, t2)):
        t = o.set_drive(body, amp, f, phase)
        if math.isfinite(off):
            o.set_drive_window(t, off)
    return o, l0


def discrete_closed_form(m, k, gamma, a, T, l0, cm, times, t1=math.inf, t2=math.inf):
    """Positions (x2, x1, x3) at the given step counts, summed in closed form."""
    Kc = np.array([[2.0, 1.0], [1.0, 2.0]])
    I2 = np.eye(2)
    Mx = np.block([[I2 - k * Kc / m, I2 - gamma * Kc / m], [-k * Kc / m, I2 - gamma * Kc / m]])
    N = np.vstack([Kc / m, Kc / m])
    lam, P = np.linalg.eig(Mx)
    Pinv = np.linalg.inv(P)
    omega = 2 * math.pi / T
    j3 = math.ceil(T / 4 - 1e-9)
    # drive pieces: (input vector for (D2, D3), phase, first step, end step)
    pieces = [(np.array([-a, 0.0]), 0.0, 0, t1), (np.array([0.0, a]), math.pi / 2, j3, t2)]
    out = []
    for n in times:
        c = np.zeros(4, dtype=complex)          # starts at rest, undeformed
        for b, phase, j0, j1 in pieces:
            J = int(min(n, j1))
            if J <= j0:
                continue
            g = Pinv @ (N @ b)
            # sum_{j=j0}^{J-1} lam^(n-1-j) sin(omega j - phase)
            for sgn in (1.0, -1.0):
                z = np.exp(1j * sgn * omega)
                rho = z / lam
                geo = (rho ** j0 - rho ** J) / (1 - rho)
                c += g * lam ** (n - 1) * geo * np.exp(-1j * sgn * phase) * (sgn / 2j)
        zq = (P @ c).real
        q1, q2 = zq[0], zq[1]
        x1 = cm - (q1 + q2) / 3.0
        out.append((x1 + q1 - l0, x1, x1 + q2 + l0))
    return np.array(out)


def test_vacuum_triplet_matches_discrete_closed_form():
    m, k, gamma, a = lattice_params()
    # the converted values: m = 400 and omega_0 / omega = 6.02
    assert abs(m - 400.0) < 1e-9
    assert abs(math.sqrt(k / m) / (2 * math.pi / T_STEPS) - 6.02) < 0.01
    t1, t2 = 140580, 147609          # switch-off times of Sec. 5.1 / Fig. 9
    o, l0 = vacuum_swimmer(m, k, gamma, a, T_STEPS, t1=t1, t2=t2)
    times = [1, 2, 3, 500, 7029, 7030, 20000, 60000, 140580, 140600, 147609, 150000, 196812]
    done = 0
    got = []
    for n in times:
        o.step(n - done)
        done = n
        got.append(o.bodies()[:, 0])
    exact = discrete_closed_form(m, k, gamma, a, T_STEPS, l0, 50.0, times, t1, t2)
    got = np.array(got)
    # deformations are O(1-10) lattice cells; positions O(50)
    assert np.abs(got - exact).max() < 1e-10 * 50
    # the swimmer returns to its rest configuration after the drive stops
    assert abs(got[-1][1] - got[-1][0] - l0) < 0.05


def continuous_amplitudes(m, k, gamma, a, omega):
    """Complex steady-state amplitudes of (x2, x1, x3) for the continuous ODE."""
    Lp = np.array([[1.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 1.0]])
    # D2 = -a sin(wt) = Re(i a e^{iwt}); D3 = a sin(wt - pi/2) = Re(-a e^{iwt})
    F2, F3 = 1j * a, -a + 0j
    F = np.array([F2, -(F2 + F3), F3])
    A = -omega ** 2 * m * np.eye(3) + 1j * omega * gamma * Lp + k * Lp
    return np.linalg.solve(A, F)


def steady_amplitude_b2(m, k, gamma, a, T, periods):
    o, _ = vacuum_swimmer(m, k, gamma, a, T)
    o.step(int((periods - 1) * T))
    xs = []
    for _ in range(int(T)):
        o.step(1)
        xs.append(o.bodies()[0, 0])
    t = np.arange(len(xs))
    w = 2 * math.pi / T
    B = np.column_stack([np.ones_like(t, dtype=float), np.cos(w * t), np.sin(w * t)])
    coef, *_ = np.linalg.lstsq(B, np.array(xs), rcond=None)
    return math.hypot(coef[1], coef[2])


def test_vacuum_steady_amplitude_matches_continuous_solution():
    """Paper's Fig. 9 parameters: simulated amplitude of sphere 2 vs analytic."""
    m, k, gamma, a = lattice_params()
    omega = 2 * math.pi / T_STEPS
    A_exact = abs(continuous_amplitudes(m, k, gamma, a, omega)[0])
    A_sim = steady_amplitude_b2(m, k, gamma, a, T_STEPS, periods=8)
    assert abs(A_sim / A_exact - 1.0) < 2e-3


def test_vacuum_resonances_at_omega0_equal_omega_and_omega_over_sqrt3():
    """Fig. 10: A/a of sphere 2 against omega_0/omega at damping ratio D = 0.07
    has maxima near omega_0 = omega / sqrt(3) (the symmetric mode sqrt(3)
    omega_0 meets omega; its larger damping pulls the peak a little lower)
    and at omega_0 = omega (the antisymmetric mode)."""
    m, T, a, D = 1.0, 400.0, 1e-4, 0.07
    omega = 2 * math.pi / T
    low = [0.45 + 0.03 * i for i in range(9)]
    high = [0.87 + 0.03 * i for i in range(10)]
    sims = {}
    for r in low + high:
        k = m * (r * omega) ** 2
        gamma = 2 * D * math.sqrt(m * k)
        exact = abs(continuous_amplitudes(m, k, gamma, a, omega)[0])
        sims[r] = steady_amplitude_b2(m, k, gamma, a, T, periods=40)
        assert abs(sims[r] / exact - 1.0) < 0.03          # O(omega dt) = 1.6e-2
    r_low = max(low, key=lambda r: sims[r])
    r_high = max(high, key=lambda r: sims[r])
    assert 0.5 <= r_low <= 1 / math.sqrt(3) + 0.01
    assert abs(r_high - 1.0) < 0.035
