"""Pin of the oracle's running velocity average (Sec. 6, the flow fields
averaged over swimming cycles): the average over n steps equals, by brute
force, the mean of the n velocity fields exported after each step (the
REF_FIELD_U value, itself pinned by the Poiseuille and duct tests), obstacle
cells included with velocity 0; restarting the average starts from zero."""
import numpy as np

import oracle
from paper_1108_0786_gb300 import workloads as wl


def swimmer():
    sc = wl.Scenario("average", 24, 20, 28, 0.9, bc=wl.PERIODIC_Z, g=(0.0, 0.0, 2e-6))
    wl.add_swimmer(sc, (11.6, 9.8, 13.7), (0.7071, 0.0, -0.7071, 0.0), (wl.SPHERE,) * 3, 2.5, 0.0,
                   7.5, 0.02, 0.01, 4e-3, 24.0, density=2.0)
    return sc


def test_average_is_the_mean_of_the_exported_fields():
    o = oracle.from_scenario(swimmer())
    for b in range(3):                       # the swimmer moves across cell centres
        st = o.bodies()[b].copy()
        st[7:10] = (0.01, -0.015, 0.04)
        o.set_body_state(b, st)
    o.step(5)
    o.average_begin()
    us, flags = [], set()
    for _ in range(37):
        o.step(1)
        us.append(o.u())
        flags.add(o.flags().tobytes())
    avg, n = o.average()
    assert n == 37
    assert len(flags) > 5, "the swimmer must move across cell centres"
    want = np.mean(us, axis=0)
    assert np.abs(avg - want).max() <= 1e-15 * np.abs(want).max()
    # a restart counts only the steps after it
    o.average_begin()
    us2 = []
    for _ in range(2):
        o.step(1)
        us2.append(o.u())
    avg2, n2 = o.average()
    assert n2 == 2
    want2 = np.mean(us2, axis=0)
    assert np.abs(avg2 - want2).max() <= 1e-15 * np.abs(want2).max()
