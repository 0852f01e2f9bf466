"""Pins of the oracle's reverse mode against central finite differences.

The oracle's adjoint returns the gradient of J = seed . (body states after n
steps) with the obstacle maps of the run held fixed.  Central differences of
the oracle's own forward run (the definition of the derivative) pin it, for
every parameter class: drive amplitude and phase (Eq. FB1-FB3), spring
constant, rest length and damping (Eq. osci_i, osci_j), body mass and moments
of inertia (Algorithm 1), the body states and populations the run starts from,
and the capsule length through mass, inertia and volume.  Every difference
pair is checked to have run through the same obstacle maps (the flag digest),
and the fluid runs are checked to uncover and cover cells, so that the
refill and moving bounce-back parts of the sweep are exercised.

The tolerance is the finite-difference error: a relative truncation part
and a rounding part of order eps |J| / h.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from adjoint_helpers import N_STEPS, SEED, scenario, start
from paper_1108_0786_gb300 import workloads as wl


def run(sc, options=0, dstate=None, dpop=None):
    o = start(sc, options, dstate)
    if dpop is not None:
        o.set_pop(o.pop() + dpop)
    o.step(N_STEPS)
    return float((o.bodies() * SEED).sum()), o.flag_digest


def central(fn, h):
    jp, dp = fn(h)
    jm, dm = fn(-h)
    assert dp == dm, "the difference step changed an obstacle map"
    return (jp - jm) / (2 * h), max(abs(jp), abs(jm))


def check(ad, fd, jmag, h, rel=5e-6):
    tol = rel * abs(fd) + 100 * 2.2e-16 * jmag / h
    assert abs(ad - fd) <= tol, (ad, fd, tol)


@pytest.fixture(scope="module", params=[oracle.OPT_NO_FLUID, 0], ids=["bodies-only", "coupled"])
def case(request):
    opts = request.param
    sc = scenario()
    o = start(sc, opts)
    f0 = o.flags()
    g = o.adjoint(N_STEPS, SEED)
    if opts == 0:
        # the run covers and uncovers cells: refill and moving walls are exercised
        assert (o.flags() != f0).sum() > 20
    return opts, g


@pytest.mark.parametrize("term,col,h", [(0, 0, 1e-6), (2, 0, 1e-6), (3, 0, 1e-6), (2, 1, 1e-5), (3, 1, 1e-5)])
def test_drive_gradient(case, term, col, h):
    opts, g = case

    def fn(e):
        sc = scenario()
        d = sc.drives[term]
        sc.drives[term] = dataclasses.replace(d, amp=d.amp + e) if col == 0 else \
            dataclasses.replace(d, phase=d.phase + e)
        return run(sc, opts)
    fd, jmag = central(fn, h)
    check(g["drive"][term, col], fd, jmag, h)


@pytest.mark.parametrize("spring,col,h", [(0, 0, 1e-6), (1, 0, 1e-6), (0, 1, 1e-5), (1, 1, 1e-5),
                                          (0, 2, 1e-5), (1, 2, 1e-5)])
def test_spring_gradient(case, spring, col, h):
    opts, g = case

    def fn(e):
        sc = scenario()
        s = sc.springs[spring]
        field = ("k", "rest", "damping")[col]
        sc.springs[spring] = dataclasses.replace(s, **{field: getattr(s, field) + e})
        return run(sc, opts)
    fd, jmag = central(fn, h)
    check(g["spring"][spring, col], fd, jmag, h)


@pytest.mark.parametrize("body", [0, 1])
def test_mass_gradient(case, body):
    """Scaling a sphere's mass scales its inertia with it: the total
    derivative is dJ/dm + sum_i dJ/dI_i * I_i / m."""
    opts, g = case
    sc = scenario()
    m = sc.bodies[body].mass
    inertia = oracle.from_scenario(sc, opts).body_props(body)[1:]
    h = 1e-6 * m

    def fn(e):
        s = scenario()
        s.bodies[body] = dataclasses.replace(s.bodies[body], mass=m + e)
        return run(s, opts)
    fd, jmag = central(fn, h)
    check(g["body"][body, 0] + (g["body"][body, 1:4] * inertia / m).sum(), fd, jmag, h)


@pytest.mark.parametrize("body,comp,h", [(0, 0, 1e-5), (1, 2, 1e-5), (2, 8, 1e-6), (1, 12, 1e-6), (2, 11, 1e-6)])
def test_initial_state_gradient(case, body, comp, h):
    opts, g = case

    def fn(e):
        d = np.zeros((3, 13))
        d[body, comp] = e
        return run(scenario(), opts, dstate=d)
    fd, jmag = central(fn, h)
    check(g["state"][body, comp], fd, jmag, h)
    assert not g["prev"].any()      # the run starts at the first step: folded into "state"


def test_population_gradient_along_a_random_direction():
    """<dJ/dG, r> against the derivative of J along r (random, seeded)."""
    sc = scenario()
    o = start(sc)
    g = o.adjoint(N_STEPS, SEED)
    r = np.random.default_rng(1108).standard_normal((19, sc.nz, sc.ny, sc.nx)) * 1e-2
    h = 1e-5
    fd, jmag = central(lambda e: run(sc, dpop=e * r), h)
    check(float((g["pop"] * r).sum()), fd, jmag, h)
    assert abs(fd) > 1e-4


def test_capsule_length_gradient_with_walls_and_body_force():
    """Capsule length l enters through mass (density x volume), inertia and
    volume (the body force g V); the cell map is held fixed, so the
    difference step must flip no cell.  Walls in y and z, periodic x."""
    kw = dict(n=24, bc=wl.PERIODIC_X, g=(2e-6, 0.0, 0.0))
    l0 = 2.0
    sc = scenario(cap_len=l0, **kw)
    o = start(sc)
    g = o.adjoint(N_STEPS, SEED)

    def props(l):
        s = scenario(cap_len=l, **kw)
        vol_inertia = oracle.from_scenario(s).body_props(2)
        return np.concatenate(([s.bodies[2].mass], vol_inertia[1:], vol_inertia[:1]))
    hp = 1e-4
    dprops = (props(l0 + hp) - props(l0 - hp)) / (2 * hp)   # d(m, I1, I2, I3, V)/dl
    ad = float((g["body"][2] * dprops).sum())
    h = 1e-6
    fd, jmag = central(lambda e: run(scenario(cap_len=l0 + e, **kw)), h)
    check(ad, fd, jmag, h, rel=2e-5)
    assert abs(g["body"][2, 4]) > 0      # the volume term is live under the body force


def test_seed_linearity_and_zero_seed():
    sc = scenario()
    g1 = start(sc).adjoint(N_STEPS, SEED)
    g2 = start(sc).adjoint(N_STEPS, 2.0 * SEED)
    g0 = start(sc).adjoint(N_STEPS, np.zeros_like(SEED))
    for key in ("state", "drive", "spring", "body"):
        np.testing.assert_allclose(g2[key], 2.0 * g1[key], rtol=1e-13, atol=1e-300)
        assert not g0[key].any()
    assert math.isfinite(float(g1["pop"].sum()))
