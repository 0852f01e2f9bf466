"""The paper's swimmer design study (Sec. 5.1-5.3, Tables 1-6) on the GPU path.

Seventeen three-body swimmers, (a)-(q), in a 100 x 100 x 200 channel, driven
by the cycling protocol of Sec. 3.3 for 7 periods (T = 28116 steps) with the
drives switched off at t1 = 5T (left body) and t2 = 5T + T/4 (the others),
run together as one ensemble (lbm_ensemble_*).  From the last full driven
cycle [4T, 5T] each swimmer's speed u_swim, the Golestanian-Ajdari speed
u_GA (Eq. V_GA, Eq. K with fitted arms, Eq. arms) and Lighthill's
efficiency (Eq. eff) are computed and set beside the paper's tables.

Readings (the paper's design pictures are not available; each choice is
derived from the printed tables):
  - "rest length" is the surface gap along the swimming axis: Table 1's
    total lengths (40 = 3 x 8 + 2 x 8 for (a)) require it;
  - capsule placement: Eq. K with the effective capsule radius 6 (the mean
    of radius 4 and half-length 8) reproduces the printed K of every design
    when (b)/(g)/(l) carry one capsule at the left body B2, (c)/(h)/(m) at
    the middle body B1, (d)/(i)/(n) at the right body B3, (e)/(j)/(o) at
    both end bodies and (f)/(k)/(p) three capsules; Table 1's totals agree;
  - perpendicular capsules lie along x, across the swimming axis z, and are
    driven along z (a body-frame drive axis);
  - physical units: dx = 1e-6 m, dt from the printed omega, the mass unit
    1.36e-15 kg (honey's density read as 1360 kg/m^3), so nu = 1/18
    (tau = 2/3), m = 400, k = 7.25e-4, gamma = 0.0873, a = 4.19e-3;
  - the channel: no-slip walls in x and y, periodic along the swimming
    axis z; the swimmer starts at the channel centre;
  - the coupling: at the paper's equal masses the bodies are 1.49 (spheres),
    0.60 (capsules) and 0.19 (large spheres) times as dense as the fluid, and
    the plain explicit coupling of Algorithm 2 drives them into growing,
    erratic motion within a period; the study therefore runs with the
    hydrodynamic load averaged over two steps (LBM_OPT_AVERAGE_FORCE), a
    standard stabiliser of explicit fluid-rigid-body coupling that the paper
    does not mention.
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

from . import analysis, workloads as wl

PERIOD = 28116
STEPS = 196812
T_OFF_LEFT = 140580          # 5 T
T_OFF_OTHERS = 147609        # 5 T + T / 4
DOMAIN = (100, 100, 200)
OMEGA_SI = 296057.86703      # rad/s: the printed lattice omega 2 pi / T over dt
SI = {"dx": 1e-6, "nu": 7.36e-5, "mass_unit": 1.36e-15, "mass": 5.44e-13, "k": 1.72965,
      "gamma": 1.57237e-7, "amp": 1.0e-5}
R_SPHERE, R_CAP, L_CAP, R_BIG = 4.0, 4.0, 8.0, 8.0
R_EFF_CAPSULE = 6.0          # effective hydrodynamic radius of a capsule in Eq. K (reading)

# body kinds at (B2, B1, B3): S sphere, P parallel capsule, N perpendicular
# capsule, Q large sphere; surface gaps (B2-B1, B1-B3)
DESIGNS = {
    "a": ("SSS", (8, 8)), "b": ("PSS", (8, 8)), "c": ("SPS", (8, 8)), "d": ("SSP", (8, 8)),
    "e": ("PSP", (8, 8)), "f": ("PPP", (8, 8)),
    "g": ("NSS", (12, 8)), "h": ("SNS", (12, 12)), "i": ("SSN", (8, 12)), "j": ("NSN", (12, 12)),
    "k": ("NNN", (16, 16)),
    "l": ("NSS", (8, 8)), "m": ("SNS", (8, 8)), "n": ("SSN", (8, 8)), "o": ("NSN", (8, 8)),
    "p": ("NNN", (8, 8)), "q": ("QQQ", (8, 8)),
}


# the paper's results per design (Tables 2, 4, 5, 6): u_swim and u_GA in
# 1e-6 lattice units per step, the error bound in %, efficiency in 1e-4
PAPER_RESULTS = {
    "a": (9.05, 8.98, 1, 10.44), "q": (2.02, 2.45, 18, 0.88),
    "b": (7.32, 7.21, 2, 7.77), "c": (6.66, 6.31, 6, 5.86), "d": (7.11, 7.16, 1, 7.37),
    "e": (5.68, 5.48, 4, 5.31), "f": (4.78, 4.50, 7, 3.69),
    "g": (6.40, 6.82, 7, 5.97), "h": (5.71, 6.50, 13, 4.24), "i": (6.23, 6.75, 8, 5.74),
    "j": (4.21, 4.66, 10, 3.08), "k": (3.69, 3.95, 7, 2.12),
    "l": (6.75, 7.66, 12, 6.47), "m": (6.30, 8.96, 30, 4.76), "n": (6.44, 7.74, 17, 5.93),
    "o": (5.05, 6.63, 24, 4.08), "p": (4.90, 6.70, 27, 3.63),
}


def markdown_table(res):
    """The results beside the paper's (u in 1e-6, efficiency in 1e-4)."""
    lines = ["| design | u_swim | paper | u_GA | paper | error % | paper | efficiency | paper | d1 | d2 | sin dphi |",
             "|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for lab in DESIGNS:
        if lab not in res:
            continue
        r, p = res[lab], PAPER_RESULTS[lab]
        lines.append(f"| ({lab}) | {r['u_swim'] * 1e6:.2f} | {p[0]:.2f} | {r['u_ga'] * 1e6:.2f} | {p[1]:.2f} | "
                     f"{r['error_pct']:.1f} | < {p[2]} | {r['efficiency'] * 1e4:.2f} | {p[3]:.2f} | "
                     f"{r['d1']:.2f} | {r['d2']:.2f} | {r['sin_dphi']:.2f} |")
    return "\n".join(lines)


def lattice_parameters():
    """The protocol's physical parameters in lattice units (dx = dt = 1)."""
    u = analysis.lattice_units(SI["dx"], PERIOD, OMEGA_SI, SI["mass_unit"])
    nu = SI["nu"] * u["viscosity"]
    return {"nu": nu, "tau": analysis.tau_from_viscosity(nu), "mass": SI["mass"] / SI["mass_unit"],
            "k": SI["k"] * u["stiffness"], "gamma": SI["gamma"] * u["damping"], "amp": SI["amp"] * u["force"],
            "omega": 2.0 * math.pi / PERIOD}


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


Q_ALONG_Z = (math.sqrt(0.5), 0.0, -math.sqrt(0.5), 0.0)     # body x axis -> world z


def _body(kind, mass, z, centre):
    """(Body, half-extent along z, effective radius) of one body kind."""
    if kind == "S":
        return wl.Body(wl.SPHERE, R_SPHERE, 0.0, mass, (centre[0], centre[1], z)), R_SPHERE, R_SPHERE
    if kind == "Q":
        return wl.Body(wl.SPHERE, R_BIG, 0.0, mass, (centre[0], centre[1], z)), R_BIG, R_BIG
    if kind == "P":
        return (wl.Body(wl.CAPSULE, R_CAP, L_CAP, mass, (centre[0], centre[1], z), Q_ALONG_Z),
                R_CAP + 0.5 * L_CAP, R_EFF_CAPSULE)
    return wl.Body(wl.CAPSULE, R_CAP, L_CAP, mass, (centre[0], centre[1], z)), R_CAP, R_EFF_CAPSULE


def design(label, domain=DOMAIN, period=PERIOD, steps=STEPS, t_off=(T_OFF_LEFT, T_OFF_OTHERS)):
    """The scenario of design `label` and its effective radii (B2, B1, B3)."""
    kinds, gaps = DESIGNS[label]
    p = lattice_parameters()
    nx, ny, nz = domain
    sc = wl.Scenario(f"design ({label})", nx, ny, nz, p["tau"], bc=wl.PERIODIC_Z, steps=steps)
    centre = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    half = [_body(k, p["mass"], 0.0, centre)[1] for k in kinds]
    z1 = centre[2]
    z2 = z1 - (gaps[0] + half[0] + half[1])
    z3 = z1 + (gaps[1] + half[1] + half[2])
    bodies, r_eff = [], []
    for kind, z in zip(kinds, (z2, z1, z3)):
        b, _, re = _body(kind, p["mass"], z, centre)
        bodies.append(b)
        r_eff.append(re)
    sc.bodies = bodies                                   # indices: 0 = B2, 1 = B1, 2 = B3
    sc.springs.append(wl.Spring(0, 1, p["k"], z1 - z2, p["gamma"]))
    sc.springs.append(wl.Spring(2, 1, p["k"], z3 - z1, p["gamma"]))
    freq, a, phase = 1.0 / period, p["amp"], 0.5 * math.pi
    axes = [tuple(_rot(b.orient).T @ np.array([0.0, 0.0, 1.0])) for b in bodies]  # swimming axis z
    t1, t2 = t_off
    sc.drives.append(wl.Drive(0, -a, freq, 0.0, t_off=t1, axis=axes[0]))
    sc.drives.append(wl.Drive(1, a, freq, 0.0, t_off=t2, axis=axes[1]))
    sc.drives.append(wl.Drive(2, a, freq, phase, t_off=t2, axis=axes[2]))
    sc.drives.append(wl.Drive(1, -a, freq, phase, t_off=t2, axis=axes[1]))
    return sc, r_eff


def drive_forces(sc, states, t0):
    """World-frame drive force on each body at steps t0, t0 + 1, ... from the
    recorded states (the drive of step t acts with the state of step t)."""
    n = len(states)
    out = np.zeros((n, len(sc.bodies), 3))
    for k, st in enumerate(states):
        t = t0 + k
        for d in sc.drives:
            w = 2.0 * math.pi * d.freq
            if t < d.phase / w or t >= d.t_off:
                continue
            out[k, d.body] += d.amp * math.sin(w * t - d.phase) * (_rot(st[d.body, 3:7]) @ np.asarray(d.axis))
    return out


def analyse(sc, r_eff, states, t0, period=PERIOD):
    """Sec. 5.3 quantities from the states of steps t0 .. t0 + period (the
    last full driven cycle): u_swim, u_GA, error (%), Lighthill efficiency."""
    p = lattice_parameters()
    z = states[:, :, 2]
    t = np.arange(t0, t0 + len(states), dtype=np.float64)
    u_swim = analysis.swimming_speed(z[:, 1], period)
    lb1, d1, p1 = analysis.fit_arm(t, z[:, 1] - z[:, 0], p["omega"])
    lb2, d2, p2 = analysis.fit_arm(t, z[:, 2] - z[:, 1], p["omega"])
    K = analysis.ga_geometric_factor(r_eff[0], r_eff[1], r_eff[2], lb1, lb2)
    u_ga = analysis.ga_velocity(K, d1, d2, p["omega"], math.sin(p1 - p2))
    # power over the cycle: drive of step t times the velocity of that step
    f = drive_forces(sc, states[:-1], t0)
    v = states[:-1, :, 7:10]
    eff = analysis.lighthill_efficiency(p["nu"], sum(r_eff), u_swim, period, f, v)
    return {"u_swim": u_swim, "u_ga": u_ga, "error_pct": 100.0 * abs((u_ga - u_swim) / u_ga),
            "efficiency": eff, "K": K, "d1": d1, "d2": d2, "sin_dphi": math.sin(p1 - p2)}


def run(labels=None, precision="f32", period=PERIOD, steps=STEPS, domain=DOMAIN, t_off=None):
    """Run the designs as one ensemble; return {label: analysis dict}."""
    from . import lbm
    labels = list(labels or DESIGNS)
    t_off = t_off or (5 * period, 5 * period + period // 4)
    built = {lab: design(lab, domain, period, steps, t_off) for lab in labels}
    lats = []
    for lab in labels:
        lat = lbm.from_scenario(built[lab][0], precision=precision, history=period + 1,
                                options=lbm.OPT_AVERAGE_FORCE)
        lats.append(lat)
    ens = lbm.Ensemble(lats)
    ens.step(5 * period)
    ens.sync()
    cycles = {lab: lat.history(period + 1) for lab, lat in zip(labels, lats)}
    if steps > 5 * period:
        ens.step(steps - 5 * period)
        ens.sync()
    out = {}
    for lab, lat in zip(labels, lats):
        sc, r_eff = built[lab]
        res = analyse(sc, r_eff, cycles[lab], 4 * period, period)
        res["final_z_B1"] = float(lat.bodies()[1, 2])
        out[lab] = res
    ens.close()
    for lat in lats:
        lat.close()
    return out


# ---- the flow field around one and three swimmers (Sec. 6, Fig. 13) ---------

FLOW_DOMAIN = (164, 164, 240)


def flow_field_scenario(swimmers=1, domain=FLOW_DOMAIN, period=PERIOD):
    """Design (a) swimmers in the Sec. 6 channel (walls in x and y, periodic
    along the swimming axis z), drives on throughout.  Reading (the paper
    does not place them): three swimmers lie side by side across the
    channel, along x at a quarter of the width apart, centred in y and z."""
    inf = float("inf")
    one, _ = design("a", domain, period, steps=0, t_off=(inf, inf))
    if swimmers == 1:
        one.name = f"one design (a) swimmer, {domain[0]}x{domain[1]}x{domain[2]} channel"
        return one
    if swimmers != 3:
        raise ValueError("the paper shows one and three swimmers")
    import copy
    import dataclasses
    sc = copy.deepcopy(one)
    sc.name = f"three design (a) swimmers, {domain[0]}x{domain[1]}x{domain[2]} channel"
    sc.bodies, sc.springs, sc.drives = [], [], []
    dx = domain[0] / 4.0
    for k, off in enumerate((-dx, 0.0, dx)):
        base = 3 * k
        for b in one.bodies:
            sc.bodies.append(dataclasses.replace(b, pos=(b.pos[0] + off, b.pos[1], b.pos[2])))
        for sp in one.springs:
            sc.springs.append(dataclasses.replace(sp, i=sp.i + base, j=sp.j + base))
        for d in one.drives:
            sc.drives.append(dataclasses.replace(d, body=d.body + base))
    return sc


def flow_field_study(swimmers=1, precision="f32", domain=FLOW_DOMAIN, period=PERIOD, cycles=5, warm_cycles=0):
    """The velocity field averaged over `cycles` swimming cycles after
    `warm_cycles` (the device-side running average, lbm_average_*): returns
    (scenario, mean velocity [3, nz, ny, nx], steps averaged, body states at
    the start and the end of the window)."""
    from . import lbm
    sc = flow_field_scenario(swimmers, domain, period)
    lat = lbm.from_scenario(sc, precision=precision, options=lbm.OPT_AVERAGE_FORCE)
    lat.step(warm_cycles * period)
    start = lat.bodies()
    lat.average_begin()
    lat.step(cycles * period)
    avg, n = lat.average()
    end = lat.bodies()
    lat.close()
    return sc, avg, n, start, end


def flow_field_summary(sc, avg, start, end, steps):
    """Scalars of an averaged field: the mean and largest |u| over the
    fluid, the mean axial velocity in the swimmers' mid-plane z, and each
    swimmer's mean speed over the window."""
    speed = np.sqrt((avg ** 2).sum(axis=0))
    nz = avg.shape[1]
    zc = int(round(np.mean([b.pos[2] for b in sc.bodies])))
    swimmers = len(sc.bodies) // 3
    v = [float((end[3 * k:3 * k + 3, 2] - start[3 * k:3 * k + 3, 2]).mean() / steps) for k in range(swimmers)]
    return {"swimmers": swimmers, "steps": int(steps), "mean_speed": float(speed.mean()),
            "max_speed": float(speed.max()), "midplane_mean_uz": float(avg[2, zc % nz].mean()),
            "swimmer_speeds": v}


def write_pgm(path, plane):
    """An 8-bit greyscale image of a 2-D array scaled to its range."""
    a = np.asarray(plane, dtype=np.float64)
    lo, hi = float(a.min()), float(a.max())
    img = np.zeros_like(a, dtype=np.uint8) if hi <= lo else ((a - lo) / (hi - lo) * 255.0).astype(np.uint8)
    with open(path, "wb") as fh:
        fh.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        fh.write(img[::-1].tobytes())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--designs", default="".join(DESIGNS))
    ap.add_argument("--json", default=None, help="write the results as JSON to this file")
    ap.add_argument("--from-json", default=None, help="format results written earlier instead of running")
    ap.add_argument("--flow-field", type=int, choices=(1, 3), default=None,
                    help="the Sec. 6 flow field of 1 or 3 swimmers averaged over five cycles instead")
    ap.add_argument("--out-prefix", default=None,
                    help="with --flow-field: write <prefix>.npy (the mean velocity in the swimmers' x-z plane, "
                         "[3, nz, nx]) and <prefix>.pgm (its magnitude)")
    args = ap.parse_args(argv)
    if args.flow_field:
        import time
        t0 = time.perf_counter()
        sc, avg, n, start, end = flow_field_study(args.flow_field, precision=args.precision)
        res = flow_field_summary(sc, avg, start, end, n)
        res["wall_s"] = round(time.perf_counter() - t0, 1)
        res["cells"] = sc.cells
        print(json.dumps(res, indent=1))
        if args.out_prefix:
            yc = int(round(sc.bodies[0].pos[1]))
            plane = avg[:, :, yc, :]
            np.save(args.out_prefix + ".npy", plane.astype(np.float32))
            write_pgm(args.out_prefix + ".pgm", np.sqrt((plane ** 2).sum(axis=0)))
        if args.json:
            with open(args.json, "w") as fh:
                json.dump(res, fh, indent=1)
        return 0
    if args.from_json:
        with open(args.from_json) as fh:
            res = json.load(fh)
    else:
        res = run(list(args.designs), precision=args.precision)
    print(json.dumps(res, indent=1))
    print(markdown_table(res))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(res, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
