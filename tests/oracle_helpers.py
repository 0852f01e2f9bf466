"""Drive the FP64 oracle from a seeded Scenario (test infrastructure)."""
import math

import numpy as np

import oracle


def oracle_from_scenario(sc, options=0):
    o = oracle.Oracle(sc.nx, sc.ny, sc.nz, sc.tau, sc.bc, sc.g, options)
    for b in sc.bodies:
        o.add_body(b.shape, b.radius, b.length, b.mass, b.pos, b.orient)
    for s in sc.springs:
        o.add_spring(s.i, s.j, s.k, s.rest, s.damping)
    for d in sc.drives:
        t = o.set_drive(d.body, d.amp, d.freq, d.phase)
        if math.isfinite(d.t_off):
            o.set_drive_window(t, d.t_off)
    return o


def lattice():
    return oracle.lattice()


def momentum(pop, e):
    """Total momentum sum_x sum_a e_a f_a(x) of a [19, ...] population array."""
    flat = pop.reshape(19, -1).sum(axis=1)
    return e.T.astype(np.float64) @ flat
