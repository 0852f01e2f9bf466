"""The region a step's remap must rewrite (Sec. 2.3, the mapping of bodies
onto the lattice), checked on the oracle's obstacle maps.

The CUDA path keeps two flag buffers, so the remap of step n overwrites the
flags of epoch n-2, and it rewrites only (i) the cube of half-width
E + REMAP_MARGIN (E = ceil(r + l/2) + 1, REMAP_MARGIN = 3) around floor(X_n)
and (ii) within it, the cells no farther than STATIC_REACH = 4 from the
integer box [floor(X_n - reach), floor(X_n + reach)] of some body.  Every
cell whose epoch flags (solid at n, solid at n-1, a pull source solid at
n-1, and the body id) differ between epochs n-2 and n must lie in both.
Bodies here move at the largest speed a step allows (0.5 lattice units on
every axis) and turn at random.  The epoch flags are derived from the
oracle's body-id maps, so nothing of the CUDA path is involved.  The worst
cells reach E + 2 and box + 3: each bound holds with one cell to spare.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import workloads as wl

REMAP_MARGIN = 3
STATIC_REACH = 4


def epoch_flags(bid_now, bid_prev):
    """Flag byte of epoch n from the body-id maps of epochs n and n-1:
    1 solid at n, 2 solid at n-1, 4 some pull source x - e_a solid at n-1
    (the 18 non-rest D3Q19 directions, periodic box)."""
    prev = bid_prev > 0
    near = np.zeros_like(prev)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx, dy, dz) == (0, 0, 0) or abs(dx) + abs(dy) + abs(dz) == 3:
                    continue
                near |= np.roll(prev, (dz, dy, dx), axis=(0, 1, 2))
    return ((bid_now > 0) * 1 + prev * 2 + near * 4).astype(np.uint8)


def run(seed, n=40, steps=12, speed=0.5):
    rng = np.random.default_rng(seed)
    bodies = [(wl.CAPSULE, 4.0, 8.0), (wl.SPHERE, 3.5, 0.0)]
    x0 = [np.array([12.3, 14.7, 11.1]), np.array([28.6, 27.2, 29.9])]
    vel = speed * rng.choice([-1.0, 1.0], size=3)
    o = oracle.Oracle(n, n, n, 1.0)
    for (shape, r, l), x in zip(bodies, x0):
        o.add_body(shape, r, l, 1e3, tuple(x))
    maps, centres = [], []
    for k in range(steps):
        cs = []
        for b, x in enumerate(x0):
            st = np.zeros(13)
            st[0:3] = x + k * vel
            q = rng.normal(size=4)
            st[3:7] = q / np.linalg.norm(q)
            o.set_body_state(b, st)
            cs.append(st[0:3].copy())
        o.step(1)                          # the step maps the state it starts from
        maps.append(o.flags().astype(np.int32))
        centres.append(cs)
    E = [math.ceil(r + 0.5 * l) + 1 for _, r, l in bodies]
    worst_cube, worst_box = -99, -99
    for k in range(3, steps):
        now = epoch_flags(maps[k], maps[k - 1])
        old = epoch_flags(maps[k - 2], maps[k - 3])
        changed = np.argwhere((now != old) | (maps[k] != maps[k - 2]))
        assert len(changed) > 0
        for z, y, x in changed:
            p = np.array([x, y, z])
            cube, box = [], []
            for b, (_, r, l) in enumerate(bodies):
                X = centres[k][b]
                d = (p - np.floor(X).astype(int) + n // 2) % n - n // 2
                cube.append(int(np.abs(d).max()) - E[b])
                lo, hi = np.floor(X - (r + 0.5 * l)), np.floor(X + (r + 0.5 * l))
                mid = 0.5 * (lo + hi)
                dv = (p - mid + n / 2) % n - n / 2 + mid          # the image nearest the box
                box.append(float(np.max(np.maximum(lo - dv, dv - hi))))
            worst_cube = max(worst_cube, min(cube))
            worst_box = max(worst_box, min(box))
    return worst_cube, worst_box


def test_first_step_map_is_the_state_it_starts_from():
    """The procedure's premise: after set_body_state and one step, flags()
    is the map of the state that was set (a sphere: the cells whose centre
    lies within r, periodic minimum image)."""
    n, r, X = 24, 3.5, np.array([10.4, 11.6, 12.2])
    o = oracle.Oracle(n, n, n, 1.0)
    o.add_body(wl.SPHERE, r, 0.0, 1e3, (5.0, 5.0, 5.0))
    o.step(1)
    st = np.zeros(13)
    st[0:3] = X
    st[3] = 1.0
    o.set_body_state(0, st)
    o.step(1)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = [(c - X[i] + n / 2) % n - n / 2 for i, c in enumerate((x, y, z))]
    inside = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 <= r * r
    assert np.array_equal(o.flags() > 0, inside)


@pytest.mark.parametrize("seed", range(4))
def test_changed_cells_lie_in_the_remap_region(seed):
    worst_cube, worst_box = run(seed)
    assert worst_cube <= REMAP_MARGIN - 1          # E + 2: one spare cell in the cube
    assert worst_box <= STATIC_REACH - 1           # box + 3: one spare cell in the reach


def test_the_bounds_are_reached():
    """At the largest speed the worst cells do reach E + 2 and box + 3, so a
    region one cell smaller on either count would miss cells."""
    worst = [run(seed) for seed in range(6)]
    assert max(w[0] for w in worst) == REMAP_MARGIN - 1
    assert max(w[1] for w in worst) == STATIC_REACH - 1
