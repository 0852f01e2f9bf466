"""GPU reverse sweep against the oracle's reverse mode and central differences.

FP64 parity: the gradients the CUDA path returns through the C ABI
(lbm_adjoint_record + lbm_adjoint_backward, checkpoints every `segment`
steps and recomputation) are compared element by element with the oracle's
plain reverse sweep on the same seeded scenario: periodic, and with walls,
Guo forcing and a capsule; segments that do not divide the run (a ragged
last segment); a run that starts after some steps.  The tolerance is 1e-9
of each array's largest magnitude (the FP64 trajectories agree to 1e-10).

FP32 storage: the same gradients within 1e-3.  The 96 x 48 x 48 gradient
study (4000 steps, 63 segments of 64; the capsule variant over one period)
is checked against central
differences of FP64 forward runs for the drive amplitude a, the phase and
the spring constant k, with steps small enough (bodies moved by ~1e-9
cells) that no cell of the obstacle maps flips.  The capsule-length
gradient (through mass and inertia) is compared with the oracle through
the autograd binding.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from adjoint_helpers import N_STEPS, SEED, scenario, set_motion, start
from paper_1108_0786_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1108_0786_gb300 import _build
    _build.build()
    return torch


def gpu_gradients(sc, precision="f64", n=N_STEPS, segment=16, pre=0, seed=SEED, want_pop=True):
    lat = set_motion(lbm.from_scenario(sc, precision=precision))
    if pre:
        lat.step(pre)
    lat.adjoint_record(n, segment)
    g = lat.adjoint_backward(seed, want_pop=want_pop)
    g["final"] = lat.bodies()
    lat.close()
    return g


def oracle_gradients(sc, n=N_STEPS, pre=0, seed=SEED):
    o = start(sc)
    if pre:
        o.step(pre)
    g = o.adjoint(n, seed)
    g["final"] = o.bodies()
    return g


def assert_close(got, ref, rel, keys=("state", "prev", "drive", "spring", "body", "pop")):
    for k in keys:
        scale = max(np.abs(ref[k]).max(), 1e-300)
        err = np.abs(got[k] - ref[k]).max()
        assert err <= rel * scale, (k, err, scale)


@pytest.mark.parametrize("variant", ["periodic", "walls-force-capsule"])
def test_fp64_gradients_match_the_oracle(gpu, variant):
    if variant == "periodic":
        sc = scenario()
    else:
        sc = scenario(bc=wl.PERIODIC_X, g=(2e-6, 0.0, 0.0), cap_len=3.0)
    got = gpu_gradients(sc)
    ref = oracle_gradients(sc)
    np.testing.assert_allclose(got["final"], ref["final"], rtol=1e-10, atol=1e-12)
    assert_close(got, ref, 1e-9)
    assert np.abs(ref["pop"]).max() > 0 and np.abs(ref["body"][:, 4]).max() >= 0


def test_segment_length_does_not_change_the_gradients(gpu):
    sc = scenario()
    ref = gpu_gradients(sc, segment=N_STEPS)
    for seg in (1, 7, 13):
        got = gpu_gradients(sc, segment=seg)
        for k in ("state", "drive", "spring", "body", "pop"):
            assert np.array_equal(got[k], ref[k]), (seg, k)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_overlapped_and_serial_recomputation_give_the_same_bits(gpu, precision):
    """Two slot sets (segment k - 1 recomputed on its own stream beside the
    reverse steps of segment k) and one (segments in turn) give the same
    gradients bit for bit; so do a second call on the same recording."""
    sc = scenario()
    lat = set_motion(lbm.from_scenario(sc, precision=precision))
    lat.adjoint_record(N_STEPS, 5)
    runs = []
    for serial in (0, 1, 0):
        lat.debug_set(lbm.DEBUG_ADJOINT_SERIAL, serial)
        runs.append(lat.adjoint_backward(SEED, want_pop=True))
    lat.close()
    for k in ("state", "prev", "drive", "spring", "body", "pop"):
        assert np.array_equal(runs[0][k], runs[1][k]), k
        assert np.array_equal(runs[0][k], runs[2][k]), k


def test_run_starting_after_some_steps(gpu):
    """n0 > 0: the state before the first recorded step is its own input."""
    sc = scenario()
    got = gpu_gradients(sc, n=40, pre=11, segment=9)
    ref = oracle_gradients(sc, n=40, pre=11)
    assert np.abs(ref["prev"]).max() > 0
    assert_close(got, ref, 1e-9)


def test_seed_on_every_state_component(gpu):
    """A dense seed (every component of every body) exercises every output."""
    sc = scenario()
    seed = np.random.default_rng(7).standard_normal((3, 13))
    got = gpu_gradients(sc, seed=seed, n=30, segment=8)
    ref = oracle_gradients(sc, seed=seed, n=30)
    assert_close(got, ref, 1e-9)


def test_fp32_gradients_close_to_fp64(gpu):
    sc = scenario()
    got = gpu_gradients(sc, precision="f32")
    ref = oracle_gradients(sc)
    assert_close(got, ref, 1e-3, keys=("state", "drive", "spring", "body"))


def test_adjoint_needs_a_recording_and_supported_storage(gpu):
    sc = scenario()
    lat = lbm.from_scenario(sc, precision="f64")
    with pytest.raises(lbm.LbmError) as e:
        lat.adjoint_backward(SEED)
    assert e.value.code == lbm.E_STATE
    lat.close()
    lat = lbm.from_scenario(sc, precision="f16")
    with pytest.raises(lbm.LbmError) as e:
        lat.adjoint_record(10, 4)
    assert e.value.code == lbm.E_ARG
    lat.close()


# ---- the 96 x 48 x 48 gradient study against central differences ----------

def design(capsules, steps, **kw):
    sc = wl.design_swimmer(capsules=capsules, steps=steps)
    for key, v in kw.items():
        if key == "a":
            sc.drives = [dataclasses.replace(d, amp=math.copysign(v, d.amp)) for d in sc.drives]
        elif key == "phase":
            sc.drives = [dataclasses.replace(d, phase=v) if d.phase > 0 else d for d in sc.drives]
        elif key == "k":
            sc.springs = [dataclasses.replace(s, k=v) for s in sc.springs]
        elif key == "l":
            sc.bodies = [dataclasses.replace(b, length=v, mass=wl.capsule_volume(b.radius, v))
                         for b in sc.bodies]
    return sc


def displacement(sc, precision="f64"):
    """x displacement of the middle body and a digest of the obstacle map
    every 64 steps (a flipped cell between two difference runs shows up in
    the digests, or as a jump the gradient check rejects)."""
    import hashlib
    lat = lbm.from_scenario(sc, precision=precision)
    x0 = lat.bodies()[1, 0]
    maps = hashlib.sha256()
    for _ in range(sc.steps // 64):
        lat.step(64)
        maps.update(lat.field(lbm.FIELD_FLAGS).tobytes())
    lat.step(sc.steps % 64)
    maps.update(lat.field(lbm.FIELD_FLAGS).tobytes())
    x = lat.bodies()[1, 0]
    lat.close()
    return x - x0, maps.hexdigest()


@pytest.mark.parametrize("precision,rel", [("f64", 2e-3), ("f32", 1e-2)])
def test_design_swimmer_gradients_against_central_differences(gpu, precision, rel):
    # the capsule swimmer loses its axial alignment after about two periods
    # (a rotational instability seeded by round-off: Omega grows from 1e-16
    # to 1e-3); past it J is too sensitive for difference quotients to
    # converge, so the capsule variant is checked over one period
    for capsules, steps in ((False, 4000), (True, 500)):
        sc = design(capsules, steps)
        lat = lbm.from_scenario(sc, precision=precision)
        seed = np.zeros((3, 13))
        seed[1, 0] = 1.0
        lat.adjoint_record(sc.steps, 64)
        g = lat.adjoint_backward(seed)
        lat.close()
        a0, ph0, k0 = 5e-4, math.pi / 2, 0.015
        signs = np.array([math.copysign(1.0, d.amp) for d in sc.drives])
        # difference steps sized to move the bodies by about 1e-9 cells
        # (larger steps flip cells of the map within 4000 steps; the FP64
        # round-off of a run limits the difference to ~1e-4 relative)
        grads = {
            "a": float((g["drive"][:, 0] * signs).sum()),
            "k": float(g["spring"][:, 0].sum()),
            # the switch-on step of the delayed terms sits on the step grid
            # (phase / omega = T / 4): difference just below it, where it is fixed
            "phase": float(sum(g["drive"][i, 1] for i, d in enumerate(sc.drives) if d.phase > 0)),
        }
        # (the capsule length acts through mass and inertia only: a step that
        # keeps the maps moves J by ~1e-14, below a run's round-off, so its
        # gradient is checked against the oracle, not by differences here)
        checks = {key: (ad, 1e-9 / max(abs(ad), 1e-6)) for key, ad in grads.items()}
        for key, (ad, h) in checks.items():
            x0 = {"a": a0, "k": k0, "phase": ph0}[key]
            if key == "phase":
                (jp, fp), (jm, fm) = displacement(design(capsules, steps, phase=x0 - h)), \
                    displacement(design(capsules, steps, phase=x0 - 3 * h))
            else:
                (jp, fp), (jm, fm) = displacement(design(capsules, steps, **{key: x0 + h})), \
                    displacement(design(capsules, steps, **{key: x0 - h}))
            assert fp == fm, f"{key}: the difference step changed an obstacle map"
            fd = (jp - jm) / (2 * h)
            assert abs(ad - fd) <= rel * abs(fd), (capsules, key, ad, fd)


def test_autograd_function_matches_the_oracle(gpu):
    """swimmer_run (torch.autograd.Function over the C ABI) against the
    oracle's reverse mode, including the chain rule of mass and capsule
    length through the inertia and volume formulas."""
    import torch
    from paper_1108_0786_gb300 import autograd as ag
    sc = scenario(bc=wl.PERIODIC_X, g=(2e-6, 0.0, 0.0), cap_len=3.0)
    p = ag.scenario_parameters(sc)
    p["state0"] = torch.from_numpy(start(sc).bodies())    # the oracle's start state, bit for bit
    for v in p.values():
        v.requires_grad_(True)
    final = ag.swimmer_run(sc, N_STEPS, segment=16, precision="f64", **p)
    (final * torch.from_numpy(SEED)).sum().backward()
    ref = oracle_gradients(sc)
    np.testing.assert_allclose(final.detach().numpy(), ref["final"], rtol=1e-10, atol=1e-12)

    def close(got, want):
        want = np.asarray(want)
        assert np.abs(got.detach().numpy() - want).max() <= 1e-9 * max(np.abs(want).max(), 1e-300)
    close(p["amp"].grad, ref["drive"][:, 0])
    close(p["phase"].grad, ref["drive"][:, 1])
    close(p["k"].grad, ref["spring"][:, 0])
    close(p["rest"].grad, ref["spring"][:, 1])
    close(p["damping"].grad, ref["spring"][:, 2])
    close(p["state0"].grad, ref["state"])
    # mass and length: the oracle's (m, I, V) gradients through differences
    # of the oracle's own body properties
    o = oracle.from_scenario(sc)
    dmass, dlen = np.zeros(3), np.zeros(3)
    for b, body in enumerate(sc.bodies):
        def props(m, l):
            s2 = dataclasses.replace(body, mass=m, length=l)
            o2 = oracle.Oracle(sc.nx, sc.ny, sc.nz, sc.tau, sc.bc, sc.g)
            o2.add_body(s2.shape, s2.radius, s2.length, s2.mass, s2.pos, s2.orient)
            vi = o2.body_props(0)
            return np.concatenate(([m], vi[1:], vi[:1]))
        hm = 1e-4 * body.mass
        dmass[b] = (ref["body"][b] * (props(body.mass + hm, body.length) - props(body.mass - hm, body.length))
                    / (2 * hm)).sum()
        if body.shape == wl.CAPSULE:
            hl = 1e-4
            dlen[b] = (ref["body"][b] * (props(body.mass, body.length + hl) - props(body.mass, body.length - hl))
                       / (2 * hl)).sum()
    assert np.abs(p["mass"].grad.numpy() - dmass).max() <= 1e-7 * np.abs(dmass).max()
    assert abs(p["length"].grad[2].item() - dlen[2]) <= 1e-7 * abs(dlen[2])
    assert dlen[2] != 0.0
    del o


def test_drive_axes_forward_and_reverse_match_the_oracle(gpu):
    """Drive terms along body-frame axes on turned bodies: FP64 trajectory
    and every gradient against the oracle."""
    from adjoint_helpers import axis_swimmer
    sc = axis_swimmer((0.8, 0.3, -0.4, 0.33), (1, 0, 0))
    seed = np.random.default_rng(11).standard_normal((3, 13))
    lat = lbm.from_scenario(sc, precision="f64")
    lat.adjoint_record(50, 16)
    got = lat.adjoint_backward(seed, want_pop=True)
    got["final"] = lat.bodies()
    lat.close()
    o = oracle.from_scenario(sc)
    ref = o.adjoint(50, seed)
    np.testing.assert_allclose(got["final"], o.bodies(), rtol=1e-10, atol=1e-12)
    assert_close(got, ref, 1e-9)
