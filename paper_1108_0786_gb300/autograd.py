"""PyTorch autograd binding of the reverse sweep.

``swimmer_run`` returns the body states after ``steps`` coupled steps of a
scenario as a differentiable function of the swimmer parameters: drive
amplitudes and phases (Eq. FB1-FB3), spring constants, rest lengths and
dampings (Eq. osci_i, osci_j), body masses, capsule lengths and the start
state of the bodies.  The forward pass runs the GPU library with a
recording (``lbm_adjoint_record``, checkpoints every ``segment`` steps); the
backward pass runs its reverse sweep (``lbm_adjoint_backward``) on the
incoming gradient of the final states.  The obstacle maps of the recorded
run are held fixed, so a capsule length acts through the body's mass
distribution (principal moments of inertia) and volume only.

Argument marshalling only: both passes run in the library's CUDA kernels.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np
import torch

from . import lbm, workloads as wl


def _scenario_with(sc, amp, phase, k, rest, damping, mass, length):
    out = copy.deepcopy(sc)
    out.drives = [dataclasses.replace(d, amp=float(a), phase=float(p))
                  for d, a, p in zip(sc.drives, amp, phase)]
    out.springs = [dataclasses.replace(s, k=float(kk), rest=float(rr), damping=float(dd))
                   for s, kk, rr, dd in zip(sc.springs, k, rest, damping)]
    out.bodies = [dataclasses.replace(b, mass=float(m), length=float(l) if b.shape == wl.CAPSULE else 0.0)
                  for b, m, l in zip(sc.bodies, mass, length)]
    return out


class _SwimmerRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amp, phase, k, rest, damping, mass, length, state0, sc, steps, segment, precision):
        run = _scenario_with(sc, amp.tolist(), phase.tolist(), k.tolist(), rest.tolist(),
                             damping.tolist(), mass.tolist(), length.tolist())
        lat = lbm.from_scenario(run, precision=precision)
        s0 = state0.detach().cpu().double().numpy()
        for b in range(len(run.bodies)):
            lat.set_body_state(b, s0[b])
        lat.adjoint_record(int(steps), int(segment))
        final = torch.from_numpy(lat.bodies())
        ctx.lat = lat
        ctx.run = run
        ctx.save_for_backward(mass, length)
        return final.to(state0.dtype)

    @staticmethod
    def backward(ctx, grad_final):
        mass, length = ctx.saved_tensors
        g = ctx.lat.adjoint_backward(grad_final.detach().cpu().double().numpy())
        ctx.lat.close()
        ctx.lat = None
        nb = len(ctx.run.bodies)
        d_mass = np.zeros(nb)
        d_length = np.zeros(nb)
        for b, body in enumerate(ctx.run.bodies):
            d_mass[b], d_length[b] = _mass_length_chain(body, float(mass[b]), float(length[b]), g["body"][b])
        t = lambda a, like: torch.as_tensor(a, dtype=like.dtype, device=like.device)
        return (t(g["drive"][:, 0], mass), t(g["drive"][:, 1], mass), t(g["spring"][:, 0], mass),
                t(g["spring"][:, 1], mass), t(g["spring"][:, 2], mass), t(d_mass, mass),
                t(d_length, length), t(g["state"], grad_final), None, None, None, None)


def _mass_length_chain(body, mass, length, gbody):
    """dJ/dm and dJ/dl from the reverse sweep's dJ/d(m, I1, I2, I3, V) and
    the library's derivatives of (V, I1, I2, I3) with respect to mass and
    length (lbm_body_properties)."""
    l = length if body.shape == wl.CAPSULE else 0.0
    _, d_m, d_l = lbm.body_properties(body.shape, body.radius, l, mass)
    # gbody is ordered (m, I1, I2, I3, V), the derivatives (V, I1, I2, I3)
    g = np.concatenate((gbody[4:5], gbody[1:4]))
    dm = float(gbody[0] + g @ d_m)
    dl = float(g @ d_l) if body.shape == wl.CAPSULE else 0.0
    return dm, dl


def swimmer_run(sc, steps, amp, phase, k, rest, damping, mass, length, state0, segment=64,
                precision="f64"):
    """Final body states [nbodies, 13] after ``steps`` steps of scenario
    ``sc`` with the given parameter tensors (CPU, float64):

    amp, phase        [ndrives]   per drive term, in the scenario's order
    k, rest, damping  [nsprings]
    mass, length      [nbodies]   (length is ignored for spheres)
    state0            [nbodies, 13] start states (lbm_get_bodies layout)

    Differentiable in every tensor argument (a unit quaternion in state0 is
    taken as given).  ``precision``: "f64" or "f32" storage."""
    return _SwimmerRun.apply(amp, phase, k, rest, damping, mass, length, state0, sc, steps, segment,
                             precision)


def scenario_parameters(sc):
    """The parameter tensors of ``swimmer_run`` for a scenario as it stands."""
    f = lambda v: torch.tensor(v, dtype=torch.float64)
    state0 = np.zeros((len(sc.bodies), 13))
    for i, b in enumerate(sc.bodies):
        state0[i, 0:3] = b.pos
        q = np.asarray(b.orient, dtype=np.float64)
        state0[i, 3:7] = q / np.linalg.norm(q)
    return dict(amp=f([d.amp for d in sc.drives]), phase=f([d.phase for d in sc.drives]),
                k=f([s.k for s in sc.springs]), rest=f([s.rest for s in sc.springs]),
                damping=f([s.damping for s in sc.springs]), mass=f([b.mass for b in sc.bodies]),
                length=f([b.length for b in sc.bodies]), state0=torch.from_numpy(state0))
