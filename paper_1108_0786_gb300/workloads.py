"""Seeded synthetic scenarios for the coupled LBM / swimmer step.

This module only generates inputs: domain sizes, body lists, springs and
drive terms, drawn from a counter-based generator (splitmix64) with fixed
seeds.  It holds none of the method's arithmetic, and both the GPU library
and the FP64 oracle are driven from the same ``Scenario`` objects.

The scenarios stand in for the paper's parameter-study workloads (Sec. 5.1:
three-body swimmers of spheres or capsules, springs of a fixed rest length,
sinusoidal drives with the third body delayed by a quarter period); the paper
uses no public dataset.  All values are in lattice units.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

SPHERE, CAPSULE = 0, 1
PERIODIC_ALL = 7
PERIODIC_X = 1
PERIODIC_Y = 2
PERIODIC_Z = 4

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): a counter-based 64-bit generator."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def choice(self, seq):
        return seq[self.next_u64() % len(seq)]

    def quaternion(self) -> Tuple[float, float, float, float]:
        """Uniformly distributed unit quaternion (Shoemake's subgroup method)."""
        u1, u2, u3 = self.uniform(), self.uniform(), self.uniform()
        a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
        return (b * math.cos(2 * math.pi * u3), a * math.sin(2 * math.pi * u2),
                a * math.cos(2 * math.pi * u2), b * math.sin(2 * math.pi * u3))


@dataclass
class Body:
    shape: int
    radius: float
    length: float
    mass: float
    pos: Tuple[float, float, float]
    orient: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 0.0)


@dataclass
class Spring:
    i: int
    j: int
    k: float
    rest: float
    damping: float


@dataclass
class Drive:
    body: int
    amp: float
    freq: float
    phase: float
    t_off: float = math.inf
    axis: Tuple[float, float, float] = (1.0, 0.0, 0.0)    # body-frame direction


@dataclass
class Scenario:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    bc: int = PERIODIC_ALL
    g: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    bodies: List[Body] = field(default_factory=list)
    springs: List[Spring] = field(default_factory=list)
    drives: List[Drive] = field(default_factory=list)
    steps: int = 0

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def sphere_volume(r: float) -> float:
    return 4.0 / 3.0 * math.pi * r ** 3


def capsule_volume(r: float, l: float) -> float:
    return math.pi * r * r * l + sphere_volume(r)


def _axis(q):
    """Body-frame x axis of the unit quaternion q = (w, x, y, z) in world frame."""
    w, x, y, z = q
    return (1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y))


def add_swimmer(sc: Scenario, centre, q, shapes, radius, length, rest, k, damping,
                amp, period, phase=math.pi / 2, density=1.0):
    """Three bodies B2 - B1 - B3 along the swimmer axis (body-frame x of q).

    B1 (middle) sits at ``centre``; B2 at centre - rest * axis, B3 at
    centre + rest * axis.  Springs S1 = (B2, B1) and S2 = (B3, B1).  The drive
    protocol of Sec. 3.3: F2 = -a sin(w t), F3 = a sin(w t - phase) switched on
    at t = phase / w, and F1 = -(F2 + F3) as two terms with the same timing.
    Returns the indices (B2, B1, B3).
    """
    ax = _axis(q)
    freq = 1.0 / period
    ids = []
    for side, shape in zip((-1.0, 0.0, 1.0), shapes):
        l = length if shape == CAPSULE else 0.0
        vol = capsule_volume(radius, l) if shape == CAPSULE else sphere_volume(radius)
        pos = tuple(centre[i] + side * rest * ax[i] for i in range(3))
        sc.bodies.append(Body(shape, radius, l, density * vol, pos, q))
        ids.append(len(sc.bodies) - 1)
    b2, b1, b3 = ids
    sc.springs.append(Spring(b2, b1, k, rest, damping))
    sc.springs.append(Spring(b3, b1, k, rest, damping))
    sc.drives.append(Drive(b2, -amp, freq, 0.0))
    sc.drives.append(Drive(b1, amp, freq, 0.0))
    sc.drives.append(Drive(b3, amp, freq, phase))
    sc.drives.append(Drive(b1, -amp, freq, phase))
    return b2, b1, b3


def three_sphere_periodic(seed: int = 1108) -> Scenario:
    """32^3 periodic box, tau = 1, one three-sphere swimmer along x.

    Spheres of radius 3 and density 1, springs of rest length 10 (centre to
    centre), k = 0.01, damping 0.005, drive amplitude 1e-4, period 400 steps,
    quarter-period delay on the third body; every body start coordinate is
    jittered by U[-0.1, 0.1]; 1000 steps.
    """
    rng = SplitMix64(seed)
    sc = Scenario("three-sphere 32^3 periodic FP64", 32, 32, 32, 1.0, steps=1000)
    add_swimmer(sc, (16.0, 16.0, 16.0), (1.0, 0.0, 0.0, 0.0), (SPHERE,) * 3, 3.0, 0.0,
                10.0, 0.01, 0.005, 1e-4, 400.0)
    for b in sc.bodies:
        b.pos = tuple(p + rng.uniform(-0.1, 0.1) for p in b.pos)
    return sc


def channel_swimmer(seed: int = 1108, periods: int = 10) -> Scenario:
    """128 x 64 x 64 channel: periodic x, no-slip walls in y and z.

    Body-force-driven duct flow with g_x = 1.438e-7 (Re = u_max 64 / nu ~ 0.1
    at tau = 1) and one three-sphere swimmer of radius 6 on the centre line:
    rest length 20, k = 0.02, damping 0.01, amplitude 5e-4, period 1000 steps,
    run for ``periods`` periods.
    """
    rng = SplitMix64(seed)
    sc = Scenario("channel swimmer 128x64x64", 128, 64, 64, 1.0, bc=PERIODIC_X,
                  g=(1.438e-7, 0.0, 0.0), steps=1000 * periods)
    add_swimmer(sc, (64.0, 31.5, 31.5), (1.0, 0.0, 0.0, 0.0), (SPHERE,) * 3, 6.0, 0.0,
                20.0, 0.02, 0.01, 5e-4, 1000.0)
    for b in sc.bodies:
        b.pos = (b.pos[0] + rng.uniform(-0.1, 0.1), b.pos[1], b.pos[2])
    return sc


def capsule_swarm(nx=512, ny=256, nz=256, swimmers=8, seed=1108, mix=False,
                  steps=2000) -> Scenario:
    """Periodic box holding ``swimmers`` three-capsule swimmers.

    Capsules of radius 4 and cylinder length 8 (or, with ``mix``, a seeded
    sphere/capsule mix with spheres of radius 4), density 1, springs of rest
    length 24 centre to centre (an 8-cell gap between parallel capsules),
    k = 0.01, damping 0.005, period 400, amplitude U[2e-4, 8e-4]; centres
    uniform in the box with non-overlap rejection, orientations uniform.
    """
    rng = SplitMix64(seed)
    sc = Scenario(f"capsule swarm {nx}x{ny}x{nz}, {swimmers} swimmers", nx, ny, nz, 1.0,
                  steps=steps)
    rest, r, l = 24.0, 4.0, 8.0
    reach = rest + r + 0.5 * l            # swimmer bounding-sphere radius
    centres = []
    attempts = 0
    while len(centres) < swimmers:
        attempts += 1
        if attempts > 100000:
            raise ValueError(f"cannot place {swimmers} swimmers in a {nx}x{ny}x{nz} box")
        c = (rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz))
        q = rng.quaternion()
        shapes = tuple(rng.choice((SPHERE, CAPSULE)) for _ in range(3)) if mix else (CAPSULE,) * 3
        amp = rng.uniform(2e-4, 8e-4)
        ok = True
        for c2 in centres:
            d2 = 0.0
            for i, n in enumerate((nx, ny, nz)):
                d = c[i] - c2[i]
                d -= n * round(d / n)
                d2 += d * d
            if d2 < (2 * reach + 8.0) ** 2:
                ok = False
                break
        if not ok:
            continue
        centres.append(c)
        add_swimmer(sc, c, q, shapes, r, l, rest, 0.01, 0.005, amp, 400.0)
    return sc


def design_swimmer(capsules: bool = False, seed: int = 1108, steps: int = 4000) -> Scenario:
    """96 x 48 x 48 periodic box with one swimmer for the gradient study.

    Spheres of radius 4, rest length 14 centre to centre, k = 0.015,
    damping 0.005, amplitude 5e-4, period 500 steps, density 1, tau = 1,
    4000 steps (8 periods).  With ``capsules``, three parallel capsules of
    radius 3 and cylinder length 4 (half-extent 5 along the axis, a 4-cell
    gap at rest 14).  The middle body starts at the box centre with every
    coordinate jittered by U[-0.1, 0.1].
    """
    rng = SplitMix64(seed)
    name = "design swimmer 96x48x48 " + ("capsules" if capsules else "spheres")
    sc = Scenario(name, 96, 48, 48, 1.0, steps=steps)
    centre = tuple(v + rng.uniform(-0.1, 0.1) for v in (48.0, 24.0, 24.0))
    if capsules:
        add_swimmer(sc, centre, (1.0, 0.0, 0.0, 0.0), (CAPSULE,) * 3, 3.0, 4.0, 14.0, 0.015, 0.005,
                    5e-4, 500.0)
    else:
        add_swimmer(sc, centre, (1.0, 0.0, 0.0, 0.0), (SPHERE,) * 3, 4.0, 0.0, 14.0, 0.015, 0.005,
                    5e-4, 500.0)
    return sc


def ensemble_members(n: int = 96, seed: int = 1108, density: float = 2.0):
    """``n`` independent periodic cubic boxes, one three-body swimmer each.

    Edge U{48, 64, 80, 96}; each body a sphere of radius 3 or a capsule of
    radius 3 and cylinder length 6 (p = 1/2), density 2 (radius-3 bodies at
    density 1 sit on the explicit coupling's rotational instability); rest
    lengths the two half-extents along the axis plus a 4-cell gap; k = 0.01,
    damping 0.005, amplitude U[1e-4, 1e-3], phase U[pi/4, 3pi/4], period in
    {200, 400, 800} and 5 periods of steps; the middle body at the box centre
    jittered by U[-0.5, 0.5], orientation uniform.
    """
    rng = SplitMix64(seed)
    out = []
    for i in range(n):
        L = rng.choice((48, 64, 80, 96))
        period = rng.choice((200, 400, 800))
        sc = Scenario(f"ensemble member {i}: {L}^3 periodic", L, L, L, 1.0, steps=5 * period)
        shapes = tuple(rng.choice((SPHERE, CAPSULE)) for _ in range(3))
        amp = rng.uniform(1e-4, 1e-3)
        phase = rng.uniform(math.pi / 4, 3 * math.pi / 4)
        q = rng.quaternion()
        centre = tuple(L / 2 + rng.uniform(-0.5, 0.5) for _ in range(3))
        half = [3.0 + (3.0 if sh == CAPSULE else 0.0) for sh in shapes]     # half-extent along the axis
        rest_a = half[0] + half[1] + 4.0
        rest_b = half[1] + half[2] + 4.0
        ax = _axis(q)
        offsets = (-rest_a, 0.0, rest_b)
        freq = 1.0 / period
        for sh, off in zip(shapes, offsets):
            l = 6.0 if sh == CAPSULE else 0.0
            vol = capsule_volume(3.0, l) if sh == CAPSULE else sphere_volume(3.0)
            pos = tuple(centre[k] + off * ax[k] for k in range(3))
            sc.bodies.append(Body(sh, 3.0, l, density * vol, pos, q))
        b2, b1, b3 = 0, 1, 2
        sc.springs.append(Spring(b2, b1, 0.01, rest_a, 0.005))
        sc.springs.append(Spring(b3, b1, 0.01, rest_b, 0.005))
        sc.drives.append(Drive(b2, -amp, freq, 0.0))
        sc.drives.append(Drive(b1, amp, freq, 0.0))
        sc.drives.append(Drive(b3, amp, freq, phase))
        sc.drives.append(Drive(b1, -amp, freq, phase))
        out.append(sc)
    return out


def scaled_copy(sc: Scenario, steps: int) -> Scenario:
    """The same scenario with a different step count."""
    import copy
    out = copy.deepcopy(sc)
    out.steps = steps
    return out
