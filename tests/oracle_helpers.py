"""Drive the FP64 oracle from a seeded Scenario (test infrastructure)."""
import numpy as np

import oracle


def oracle_from_scenario(sc, options=0):
    return oracle.from_scenario(sc, options)


def lattice():
    return oracle.lattice()


def momentum(pop, e):
    """Total momentum sum_x sum_a e_a f_a(x) of a [19, ...] population array."""
    flat = pop.reshape(19, -1).sum(axis=1)
    return e.T.astype(np.float64) @ flat
