"""The three-body scenario the reverse-mode tests share (oracle pins and GPU
parity): two spheres and a tilted capsule joined by two springs, moving and
turning from the first step so that cells are covered and uncovered."""
import dataclasses

import numpy as np

from paper_1108_0786_gb300 import workloads as wl

N_STEPS = 60
FREQ = 1.0 / 60.0
SEED = np.zeros((3, 13))
SEED[1, 0] = 1.0        # x of the middle body
SEED[2, 1] = 0.7        # y of the capsule
SEED[0, 10] = 3.0       # Omega_x of the first body
SEED[2, 4] = 2.0        # quaternion x of the capsule
V0 = ((0.02, 0.01, -0.004), (-0.01, 0.015, 0.0), (0.0, -0.012, 0.02))
W0 = ((0.0, 0.0, 0.003), (0.002, 0.0, 0.0), (0.0, 0.004, -0.002))


def scenario(n=24, bc=7, g=(0.0, 0.0, 0.0), amp=4e-3, phase=1.3, k=0.02, rest=7.0, gamma=0.01,
             cap_len=2.0, cap_density=2.0):
    """Two spheres and a tilted capsule joined by two springs, with the four
    drive terms of the cycling strategy (Sec. 3.3) at a phase off the step
    grid (the switch-on time phase / omega is not an integer)."""
    sc = wl.Scenario("adjoint pins", n, n, n, 0.8, bc=bc, g=g)
    r = 2.2
    m = 2.0 * wl.sphere_volume(r)
    c = n / 2
    sc.bodies.append(wl.Body(wl.SPHERE, r, 0.0, m, (c - rest + 0.3, c + 0.2, c - 0.1)))
    sc.bodies.append(wl.Body(wl.SPHERE, r, 0.0, m, (c + 0.3, c + 0.2, c - 0.1)))
    sc.bodies.append(wl.Body(wl.CAPSULE, 1.8, cap_len, cap_density * wl.capsule_volume(1.8, cap_len),
                             (c + rest + 0.3, c + 0.1, c + 0.2), (0.95, 0.1, 0.2, 0.05)))
    sc.springs.append(wl.Spring(0, 1, k, rest, gamma))
    sc.springs.append(wl.Spring(1, 2, k, rest, gamma))
    sc.drives.append(wl.Drive(0, -amp, FREQ, 0.0))
    sc.drives.append(wl.Drive(1, amp, FREQ, 0.0))
    sc.drives.append(wl.Drive(2, amp, FREQ, phase))
    sc.drives.append(wl.Drive(1, -amp, FREQ, phase))
    return sc


def set_motion(o, dstate=None):
    """Give the bodies of an oracle or a lattice their start velocities."""
    st = o.bodies()
    for b in range(3):
        st[b, 7:10] = V0[b]
        st[b, 10:13] = W0[b]
    if dstate is not None:
        st = st + dstate
    for b in range(3):
        o.set_body_state(b, st[b])
    return o


def start(sc, options=0, dstate=None):
    """An oracle at the scenario's start, bodies moving and turning."""
    import oracle
    return set_motion(oracle.from_scenario(sc, options), dstate)




def rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def axis_swimmer(q, axis_world, n=32):
    """Three spheres along x with the four drive terms; every body turned by
    q and driven along the body-frame axis that q maps to axis_world."""
    q = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    a = rot(q).T @ np.asarray(axis_world, dtype=np.float64)
    sc = wl.Scenario("axis", n, n, n, 0.9)
    m = 2.0 * wl.sphere_volume(2.5)
    for x in (n / 2 - 8.2, n / 2 + 0.1, n / 2 + 8.3):
        sc.bodies.append(wl.Body(wl.SPHERE, 2.5, 0.0, m, (x, n / 2 + 0.2, n / 2 - 0.3), tuple(q)))
    sc.springs += [wl.Spring(0, 1, 0.02, 8.3, 0.01), wl.Spring(2, 1, 0.02, 8.2, 0.01)]
    amp, f = 3e-3, 1 / 50.0
    sc.drives += [wl.Drive(0, -amp, f, 0.0, axis=tuple(a)), wl.Drive(1, amp, f, 0.0, axis=tuple(a)),
                  wl.Drive(2, amp, f, 1.1, axis=tuple(a)), wl.Drive(1, -amp, f, 1.1, axis=tuple(a))]
    return sc
