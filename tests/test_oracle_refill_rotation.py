"""Pins of the oracle's refill of uncovered cells (Sec. 2.3) and of the
rotational half of its rigid-body step (Algorithm 1, time integration).

(a) Galilean invariance through remaps.  A fluid at uniform velocity V and
    density 1 with rigid bodies translating at the same V is an exact
    steady state of the discrete method: moving bounce-back returns
    f_eq(1, V) for f_eq(1, V) (the odd part of the equilibrium is
    6 w_a e_a.V), the refill of an uncovered cell gives f_eq(1, V) (every
    neighbour has density 1 and the surface moves at V), and the link
    forces cancel in opposite pairs because a closed body has as many links
    along e_a as along -e_a, on the same lattice lines.  So every fluid
    population stays f_eq(1, V) and F = T = 0 to round-off while the bodies
    cover and uncover cells.
(b) The state that refills a cell.  After an impulsive change of a body's
    state, each uncovered cell carries the velocity of the surface of the new
    state at its centre, V + Omega x (x - X), and the density of its
    neighbours that are fluid in both epochs (the mean of their sum of
    populations before the step).
(c) Torque-free rotation.  With no fluid and no torque the angular velocity
    stays constant and the renormalised first-order quaternion update is an
    exact rotation by 2 atan(|Omega|/2) per step about Omega, applied in the
    world frame: q_n = (cos(n th/2), sin(n th/2) Omega/|Omega|) (x) q_0.
(d) The world-frame inertia.  For an axisymmetric body the change of the
    angular velocity in one step is T_axial / I_1 along the body axis and
    T_across / I_2 across it, whatever the orientation, with T the
    hydrodynamic torque the step exports and I_1, I_2 the principal moments.

Each pin is also run on copies of the oracle compiled with one mistake of
the kind it is there to catch, and must fail on every one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle_helpers import planted
from paper_1108_0786_gb300 import workloads as wl

E, W = oracle.lattice()


def qmul(a, b):
    """Hamilton product of quaternions (w, x, y, z)."""
    aw, av = a[0], np.asarray(a[1:])
    bw, bv = b[0], np.asarray(b[1:])
    return np.concatenate([[aw * bw - av @ bv], aw * bv + bw * av + np.cross(av, bv)])


def rotation(q):
    """Rotation matrix of a unit quaternion (columns: body axes in the world)."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def state(pos, q, v, om):
    return np.concatenate([pos, q, v, om]).astype(np.float64)


# ---- (a) Galilean invariance --------------------------------------------------

def check_galilean(lib=None, steps=60):
    n = 24
    V = np.array([0.045, -0.03, 0.02])
    o = oracle.Oracle(n, n, n, 0.8, lib=lib)
    qcap = np.array([0.82, 0.31, -0.36, 0.33])
    qcap /= np.linalg.norm(qcap)
    bodies = [(wl.SPHERE, 3.2, 0.0, (6.3, 7.1, 8.4), (1.0, 0.0, 0.0, 0.0)),
              (wl.CAPSULE, 2.6, 5.0, (16.2, 15.7, 14.9), tuple(qcap))]
    for shape, r, l, pos, q in bodies:
        b = o.add_body(shape, r, l, 1e12, pos, q)
        o.set_body_state(b, state(pos, q, V, (0.0, 0.0, 0.0)))
    feq = oracle.equilibrium(1.0, V)
    o.set_pop(np.broadcast_to(feq[:, None, None, None], (19, n, n, n)).copy())
    changed = 0
    prev = None
    for _ in range(steps):
        o.step(1)
        flags = o.flags()
        if prev is not None:
            changed += int((flags != prev).sum())
        prev = flags
        fluid = flags == 0
        dev = np.abs(o.pop()[:, fluid] - feq[:, None]).max()
        assert dev < 1e-14, f"populations left f_eq(1, V) by {dev:.3e}"
        ft = np.abs(o.forces()).max()
        assert ft < 1e-12, f"force or torque {ft:.3e} on bodies at rest relative to the fluid"
    xb = o.bodies()
    assert np.abs(xb[:, 7:10] - V).max() < 1e-20
    assert changed > 50, "the bodies must cover and uncover cells"


def test_galilean_comoving_bodies_keep_uniform_equilibrium_through_remaps():
    check_galilean()


# ---- (b) the state that refills an uncovered cell -------------------------------

def random_pop(shape, seed, amp=2e-3):
    rng = wl.SplitMix64(seed)
    nz, ny, nx = shape
    noise = np.array([rng.uniform(-amp, amp) for _ in range(19 * nx * ny * nz)])
    return W[:, None, None, None] * (1.0 + noise.reshape(19, nz, ny, nx))


def check_refill_state(lib=None):
    n = 14
    o = oracle.Oracle(n, n, n, 0.9, lib=lib)
    X0 = np.array([6.6, 7.2, 6.9])
    q0 = np.array([1.0, 0.0, 0.0, 0.0])
    o.add_body(wl.SPHERE, 3.1, 0.0, 1e3, X0, q0)
    o.set_pop(random_pop(o.shape, 1108))
    o.step(1)
    flags0, rho0 = o.flags(), o.rho()
    # impulsive change: a new position, velocity and spin
    X1 = X0 + np.array([0.9, -0.7, 0.4])
    V1 = np.array([0.03, -0.02, 0.01])
    Om1 = np.array([0.01, -0.02, 0.015])
    o.set_body_state(0, state(X1, q0, V1, Om1))
    o.step(1)
    flags1, rho1, u1 = o.flags(), o.rho(), o.u()
    uncovered = np.argwhere((flags0 > 0) & (flags1 == 0))
    assert len(uncovered) >= 8
    both_fluid = (flags0 == 0) & (flags1 == 0)
    mixed = 0
    for z, y, x in uncovered:
        d = np.array([x, y, z], dtype=float) - X1
        d -= n * np.rint(d / n)
        uw = V1 + np.cross(Om1, d)
        assert np.abs(u1[:, z, y, x] - uw).max() < 1e-15, "refill velocity is not the new surface velocity"
        dens = []
        for a in range(1, 19):
            zz, yy, xx = (z + E[a, 2]) % n, (y + E[a, 1]) % n, (x + E[a, 0]) % n
            if both_fluid[zz, yy, xx]:
                dens.append(rho0[zz, yy, xx])
            elif flags0[zz, yy, xx] > 0 and flags1[zz, yy, xx] == 0:
                mixed += 1
        assert dens, "every uncovered cell here has fluid neighbours"
        assert abs(rho1[z, y, x] - np.mean(dens)) < 1e-15, "refill density is not the neighbours' mean"
    assert mixed > 0, "some uncovered cells must neighbour other uncovered cells"


def test_uncovered_cells_take_the_new_surface_velocity_and_the_neighbours_density():
    check_refill_state()


# ---- (c) torque-free rotation -------------------------------------------------

def check_free_rotation(lib=None, steps=400):
    o = oracle.Oracle(1, 1, 1, 1.0, options=oracle.OPT_NO_FLUID, lib=lib)
    q0 = np.array([0.6, -0.2, 0.7, 0.33])
    q0 /= np.linalg.norm(q0)
    Om = np.array([0.013, -0.021, 0.034])
    o.add_body(wl.CAPSULE, 2.0, 6.0, 50.0, (0.0, 0.0, 0.0), q0)
    o.set_body_state(0, state((0.0, 0.0, 0.0), q0, (0.0, 0.0, 0.0), Om))
    w = np.linalg.norm(Om)
    th = 2.0 * math.atan(0.5 * w)
    axis = Om / w
    for k in range(1, steps + 1):
        o.step(1)
        s = o.bodies()[0]
        r = np.concatenate([[math.cos(0.5 * k * th)], math.sin(0.5 * k * th) * axis])
        q = qmul(r, q0)
        if q @ s[3:7] < 0:
            q = -q
        assert np.abs(s[3:7] - q).max() < 1e-12, f"step {k}: quaternion off the exact rotation"
        assert np.array_equal(s[10:13], Om), "angular velocity changed without torque"


def test_torque_free_rotation_follows_the_exact_renormalised_update():
    check_free_rotation()


# ---- (d) world-frame inertia --------------------------------------------------

def check_world_inertia(lib=None, steps=12):
    n = 22
    o = oracle.Oracle(n, n, n, 1.0, lib=lib)
    q0 = np.array(wl.SplitMix64(31).quaternion())
    r, l = 3.0, 6.0
    b = o.add_body(wl.CAPSULE, r, l, wl.capsule_volume(r, l), (10.7, 11.2, 10.4), q0)
    R = rotation(q0)
    a, p = R[:, 0], R[:, 1]
    o.set_body_state(b, state((10.7, 11.2, 10.4), q0, (0.0, 0.0, 0.0), 0.004 * a + 0.003 * p))
    _, I1, I2, I3 = o.body_props(b)
    assert I2 == I3 and I1 != I2
    for _ in range(steps):
        s0 = o.bodies()[0]
        o.step(1)
        s1 = o.bodies()[0]
        T = o.forces()[0, 3:]
        ax = rotation(s0[3:7])[:, 0]
        dOm = s1[10:13] - s0[10:13]
        Ta = (ax @ T) * ax
        expect = Ta / I1 + (T - Ta) / I2
        assert np.linalg.norm(T - Ta) > 0.05 * np.linalg.norm(T), "torque must have both parts"
        err = np.abs(dOm - expect).max()
        assert err < 1e-12 * np.abs(expect).max() + 1e-22, f"change of Omega off by {err:.3e}"


def test_axisymmetric_body_turns_with_axial_and_transverse_inertia():
    check_world_inertia()


# ---- planted mistakes ---------------------------------------------------------

MISTAKES = [
    # refill velocity taken from the state before the step
    ("refill", "wall_velocity(h, &h->body[h->bid_prev[c]], p, uw);",
     "wall_velocity(h, &h->body_prev[h->bid_prev[c]], p, uw);", [check_refill_state]),
    # refill at rest instead of the surface velocity
    ("refill", "wall_velocity(h, &h->body[h->bid_prev[c]], p, uw);",
     "uw[0] = uw[1] = uw[2] = 0.0;", [check_galilean, check_refill_state]),
    # neighbours that are fluid in the current epoch only
    ("refill", "if (n < 0 || h->bid_prev[n] >= 0 || h->bid_now[n] >= 0) continue;",
     "if (n < 0 || h->bid_now[n] >= 0) continue;", [check_refill_state]),
    # refill density from the pre-collision populations
    ("refill", "for (int b = 0; b < Q; ++b) rho += h->G[b * C + n];",
     "for (int b = 0; b < Q; ++b) rho += h->F[b * C + n];", [check_refill_state]),
    # moving bounce-back along e_a instead of e_abar
    ("stream", "double eu = EX[ab] * uw[0] + EY[ab] * uw[1] + EZ[ab] * uw[2];\n"
               "                        F[ab * C + c]",
     "double eu = EX[a] * uw[0] + EY[a] * uw[1] + EZ[a] * uw[2];\n"
     "                        F[ab * C + c]", [check_galilean]),
    # momentum exchange with the wall term's sign flipped
    ("force", "double mag = 2.0 * h->G[a * C + c] + 6.0 * W[a] * rho * eu;",
     "double mag = 2.0 * h->G[a * C + c] - 6.0 * W[a] * rho * eu;", [check_galilean]),
    # torque taken to the body frame with R instead of R^T
    ("rotation", "Tb[i] = R[0][i] * Tq[k][0] + R[1][i] * Tq[k][1] + R[2][i] * Tq[k][2];",
     "Tb[i] = R[i][0] * Tq[k][0] + R[i][1] * Tq[k][1] + R[i][2] * Tq[k][2];", [check_world_inertia]),
    # principal moments applied to the wrong body axes
    ("rotation", "for (int i = 0; i < 3; ++i) Tb[i] /= b->inertia[i];",
     "for (int i = 0; i < 3; ++i) Tb[i] /= b->inertia[2 - i];", [check_world_inertia]),
    # angular velocity applied in the body frame: q += 1/2 q (x) (0, Omega)
    ("rotation", "cross(b->Om, v, c);", "cross(v, b->Om, c);", [check_free_rotation]),
    # quaternion rate without the factor 1/2
    ("rotation", "0.5 * (w * b->Om[0] + c[0]),", "(w * b->Om[0] + c[0]),", [check_free_rotation]),
]


@pytest.mark.parametrize("part,old,new,checks", MISTAKES,
                         ids=[f"{m[0]}-{i}" for i, m in enumerate(MISTAKES)])
def test_pins_fail_on_planted_mistakes(part, old, new, checks):
    lib = planted(old, new)
    for check in checks:
        with pytest.raises(AssertionError):
            check(lib)
