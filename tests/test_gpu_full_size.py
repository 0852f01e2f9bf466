"""Parity at the benchmark's full size: the 512 x 256 x 256 capsule swarm
(33.5 M cells, 24 capsules, 8 swimmers) against the FP64 oracle run on the
host cores from the same seeded state.

The bodies start with velocities of 0.15 cells a step in seeded directions,
so that over the 16 steps (one graph-launched chunk) every body covers and
uncovers cells: the remap, refill, moving bounce-back and momentum
exchange all act at full size.  Checked:
  - FP64 storage: obstacle maps bit for bit, body states to 1e-10 relative,
    forces, and the post-collision populations of a sample of cells (every
    body cell and its neighbours, plus 2^20 seeded random cells) to 1e-12;
  - FP32 storage in the launch configuration bench.py times (bulk kernel of
    2 cells a thread, at least 4 blocks per SM, graph-launched steps): maps
    bit for bit, the velocity field to 1e-5 relative L2 (the FP32 bar),
    body states to 1e-7 and the sampled populations to 1e-6.
The oracle needs ~11 GB of host memory and ~10 s on 16 cores.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1108_0786_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 16
SAMPLE = 1 << 20


@pytest.fixture(scope="module")
def reference():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    try:
        host_bytes = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        host_bytes = 0
    if host_bytes and host_bytes < 48 << 30:
        pytest.skip("the full-size oracle run needs ~32 GB of host memory")
    from paper_1108_0786_gb300 import _build
    _build.build()
    sc = wl.capsule_swarm(steps=STEPS)
    rng = np.random.default_rng(1108)
    states = []
    o = oracle.from_scenario(sc)
    st0 = o.bodies()
    for b in range(len(sc.bodies)):
        s = st0[b].copy()
        d = rng.normal(size=3)
        s[7:10] = 0.15 * d / np.linalg.norm(d)
        s[10:13] = 2e-3 * rng.normal(size=3)
        states.append(s)
        o.set_body_state(b, s)
    o.step(STEPS)
    flags = o.flags().reshape(-1).copy()
    # the sample: every body cell with its neighbours up to two cells away
    # along x and one along y and z (the link, bounce-back and refilled
    # cells among them), plus seeded random cells
    solid = np.flatnonzero(flags)
    nx, nxy, C = sc.nx, sc.nx * sc.ny, flags.size
    offs = [dx + dy * nx + dz * nxy for dx in range(-2, 3) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]
    near = np.unique(np.concatenate([(solid + o_) % C for o_ in offs]))
    rand = rng.choice(C, size=SAMPLE, replace=False)
    cells = np.unique(np.concatenate([near, rand]))
    pop = o.pop().reshape(19, -1)
    ref = {"sc": sc, "states": states, "flags": flags, "cells": cells, "pop": pop[:, cells].copy(),
           "bodies": o.bodies(), "forces": o.forces(), "u": o.u().astype(np.float64)}
    del pop
    o.close()
    assert solid.size > 0
    return ref


def gpu_run(ref, precision, shape=None):
    lat = lbm.from_scenario(ref["sc"], precision=precision)
    if shape:
        lat.tune(*shape)
    for b, s in enumerate(ref["states"]):
        lat.set_body_state(b, s)
    lat.step(STEPS)
    lat.sync()
    out = {"flags": lat.flags().reshape(-1), "bodies": lat.bodies(), "forces": lat.forces()}
    pop = lat.pop().reshape(19, -1)
    out["pop"] = pop[:, ref["cells"]].copy()
    del pop
    out["u"] = lat.u()
    lat.close()
    return out


def test_full_size_fp64_against_the_oracle(reference):
    got = gpu_run(reference, "f64")
    assert np.array_equal(got["flags"], reference["flags"])
    xb = reference["bodies"]
    assert np.abs(got["bodies"] - xb).max() <= 1e-10 * np.abs(xb[:, :3]).max()
    f = reference["forces"]
    assert np.abs(got["forces"] - f).max() <= 1e-10 * np.abs(f).max() + 1e-14
    assert np.abs(got["pop"] - reference["pop"]).max() <= 1e-12


def test_full_size_fp32_in_the_benchmark_configuration(reference):
    got = gpu_run(reference, "f32", shape=(2, 4))
    assert np.array_equal(got["flags"], reference["flags"])
    ur = reference["u"]
    assert np.linalg.norm(got["u"] - ur) <= 1e-5 * np.linalg.norm(ur)
    assert np.abs(got["bodies"] - reference["bodies"]).max() <= 1e-7
    f = reference["forces"]
    assert np.abs(got["forces"] - f).max() <= 1e-5 * np.abs(f).max()
    assert np.abs(got["pop"] - reference["pop"]).max() <= 1e-6
