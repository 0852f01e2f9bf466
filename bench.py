"""Throughput of the coupled D3Q19 LBM / rigid-body swimmer step on GB300.

One step is one pass of the whole hot path (remap, fused stream + bounce-back
+ refill + LBGK, link lists, momentum exchange, drive + springs + rigid-body
integration) over the capsule-swarm workload: a 512 x 256 x 256 periodic box
(33.5 M cells) holding 8 seeded three-capsule swimmers (capsules of radius 4
and cylinder length 8), FP32 deviation storage.  The metric is coupled-step
MLUPS (cells x steps / s / 1e6, solid cells included).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own seeded replica of the
workload (weak scaling, no data-path collective); rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS & % HBM roofline (FP32 vs FP16-store); adjoint/forward time"
UNIT = "MLUPS"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "stream_collide_capsule_swarm_traffic.txt")
KERNEL_SRC = os.path.join(ROOT, "paper_1108_0786_gb300", "csrc", "stream_collide.cu")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", default="f32", choices=("f32", "f16", "bf16", "f64"))
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--no-variants", action="store_true", help="skip the other storage precisions")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-only", action="store_true",
                    help="time only the oracle CPU baseline (no GPU) and print it as one JSON line")
    ap.add_argument("--cpu-full", action="store_true",
                    help="with --cpu-only: every config at its full step count")
    ap.add_argument("--overlap", action="store_true",
                    help="overlapped steps (the bulk kernel's far tiles beside the force and remap)")
    ap.add_argument("--shape", default="auto",
                    help="bulk-kernel shape 'cells_per_thread,min_blocks_per_sm', or 'auto' for the autotuner")
    ap.add_argument("--only", choices=("ensemble", "adjoint"), default=None,
                    help="run only the 96-box ensemble or the reverse-mode study and print its object")
    return ap.parse_args()


# ---- distributed plumbing ------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks --------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for _, _, flags in rows for n, f in zip(names, flags) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---- helpers ---------------------------------------------------------------

def hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    with open(KERNEL_SRC, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def recorded_traffic(cells):
    """DRAM bytes per stream-collide launch from the committed ncu summary,
    scaled to ``cells``; None if the kernel source changed since."""
    try:
        vals = {}
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != kernel_hash():
            return None
        return float(vals["dram_bytes_per_cell"]) * cells
    except (OSError, KeyError, ValueError):
        return None


def workload(args, rank):
    from paper_1108_0786_gb300 import workloads as wl
    return wl.capsule_swarm(nx=args.nx, ny=args.ny, nz=args.nz, swimmers=8, seed=1108 + rank,
                            steps=args.steps)


def job_mlups(cells_per_rank, steps, world, max_ms):
    """Whole-job throughput: the cells all ranks advanced per second / 1e6,
    over the slowest rank's time (weak scaling: every rank holds a replica)."""
    return cells_per_rank * steps * world / (max_ms / 1e3) / 1e6


def timed_steps(lat, steps, world, device):
    import torch
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    lat.step(steps)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    lat.sync()
    return max_over_ranks(start.elapsed_time(end), world, device)


def e2e_run(sc, args, world, device):
    """The same metric end to end through the C ABI with host buffers: the
    initial populations are uploaded from pinned host memory (lbm_set_fields)
    and every step's body states are read back into pinned host memory
    (lbm_get_bodies_async) and consumed on the host; each read is waited for
    (lbm_wait_ticket) one step later, while the next step runs."""
    import numpy as np
    import torch
    from paper_1108_0786_gb300 import lbm
    lat = lbm.from_scenario(sc, precision=args.precision)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)     # the fluid at rest
    pinned = torch.empty((19, sc.cells), dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.from_numpy(w)[:, None].expand(19, sc.cells))
    host_pop = pinned.numpy()
    lat.step(1)
    lat.sync()
    bufs = [torch.empty((lat.nbodies, 13), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    steps = args.steps
    checksum = 0.0
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.set_pop(host_pop)
    prev = None
    for k in range(steps):
        lat.step(1)
        t = lat.bodies_async(bufs[k & 1])
        if prev is not None:
            lat.wait(prev)                              # step k - 1's states are on the host
            checksum += float(bufs[(k - 1) & 1][:, 0].sum())
        prev = t
    lat.wait(prev)
    checksum += float(bufs[(steps - 1) & 1][:, 0].sum())
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world, device)
    value = sc.cells * steps * world / (ms / 1e3) / 1e6
    h2d = 19 * sc.cells * 8 / steps
    d2h = bufs[0].nbytes + 4                            # body states and the status word
    lat.close()
    del pinned, bufs
    if not np.isfinite(checksum):
        raise SystemExit("non-finite body states in the end-to-end run")
    return {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h),
            "note": "lbm_set_fields from pinned host memory once (FP64, amortised over the steps), then per "
                    "step lbm_step(1) + lbm_get_bodies_async into pinned host memory, each read waited for "
                    "(lbm_wait_ticket) and consumed on the host one step later while the next step runs"}


def swimmer_displacements(x, x0, sc):
    """Net displacement of each three-body swimmer: the mean of its bodies'."""
    import numpy as np
    d = x - x0
    return np.array([d[3 * i:3 * i + 3].mean(axis=0) for i in range(len(sc.bodies) // 3)])


def variant_runs(sc, steps):
    """Throughput of each storage precision, and its error against the FP64
    GPU path (which matches the oracle to 1e-12 in populations and 1e-10 in
    trajectories) after the workload's full step count: the relative L2
    error of the velocity field and the error of each swimmer's net
    displacement relative to the largest one."""
    import numpy as np
    from paper_1108_0786_gb300 import lbm
    res = {}
    ref = lbm.from_scenario(sc, precision="f64")
    x0 = ref.bodies()[:, :3].copy()
    ref.step(steps)
    ref_u = ref.u()
    ref_x = ref.bodies()[:, :3]
    ref_net = swimmer_displacements(ref_x, x0, sc)
    for prec in ("f32", "f16", "bf16", "f64"):
        lat = lbm.from_scenario(sc, precision=prec) if prec != "f64" else None
        if lat is not None:
            lat.step(1)
            lat.autotune(3)
            lat.step(steps - 1)
            u = lat.u()
            net = swimmer_displacements(lat.bodies()[:, :3], x0, sc)
            disp_err = float(np.linalg.norm(net - ref_net, axis=1).max() / np.linalg.norm(ref_net, axis=1).max())
            u_err = float(np.linalg.norm(u - ref_u) / np.linalg.norm(ref_u))
        else:
            lat, disp_err, u_err = ref, 0.0, 0.0
        lat.step(10)
        lat.sync()
        # eager launches: a launch the host thread was late to issue (the
        # oracle's ensemble runs share the host cores) counts its wait, so
        # the fastest of four means is taken
        ms_k = min(lat.time_kernels(5)["stream_collide"] for _ in range(4))
        t = timed_steps(lat, 200, 1, None)
        res[prec] = {"mlups": round(sc.cells * 200 / (t / 1e3) / 1e6, 1),
                     "stream_collide_gbs": round(lat.bytes_per_cell * sc.cells / (ms_k / 1e3) / 1e9, 1),
                     "bytes_per_cell": lat.bytes_per_cell,
                     "u_rel_l2_vs_f64": u_err, "net_displacement_rel_err_vs_f64": disp_err,
                     "net_displacement_abs_err_lu": float(np.linalg.norm(net - ref_net, axis=1).max())
                     if prec != "f64" else 0.0,
                     "error_after_steps": steps,
                     "error_reference": "FP64 storage on the GPU (oracle-pinned)"}
        lat.close()
    res["largest_net_displacement_lu"] = float(np.linalg.norm(ref_net, axis=1).max())
    res["channel_swimmer"] = channel_errors()
    return res


def channel_errors():
    """Each storage precision's error on the channel swimmer (128 x 64 x 64,
    walls in y and z, body-force-driven duct flow, spheres of radius 6, ten
    drive periods), the workload of the displacement bars, against the FP64
    GPU path: the relative L2 error of the velocity field and the relative
    error of the swimmer's net displacement."""
    import numpy as np
    from paper_1108_0786_gb300 import lbm, workloads as wl
    sc = wl.channel_swimmer()
    ref = lbm.from_scenario(sc, precision="f64")
    x0 = ref.bodies()[:, :3].copy()
    ref.step(sc.steps)
    ref_u = ref.u()
    ref_net = (ref.bodies()[:, :3] - x0).mean(axis=0)
    ref.close()
    out = {"steps": sc.steps, "net_displacement_lu": float(np.linalg.norm(ref_net))}
    for prec in ("f32", "f16", "bf16"):
        lat = lbm.from_scenario(sc, precision=prec)
        lat.step(sc.steps)
        net = (lat.bodies()[:, :3] - x0).mean(axis=0)
        out[prec] = {"u_rel_l2": float(np.linalg.norm(lat.u() - ref_u) / np.linalg.norm(ref_u)),
                     "net_displacement_rel_err": float(np.linalg.norm(net - ref_net) / np.linalg.norm(ref_net))}
        lat.close()
    return out


# the oracle's timed samples: (config, steps at all threads, steps at 1 thread,
# the config's full step count); configs 1 and 5 and the channel of config 2
# are the parity and gradient workloads, config 3 the benchmark's own
CPU_SAMPLES = (("three-sphere 32^3 periodic (1000 steps)", 1000, 1000, 1000),
               ("channel swimmer 128x64x64 (10 periods)", 200, 60, 10000),
               ("capsule swarm {nx}x{ny}x{nz} (8 swimmers)", 3, 1, 2000),
               ("design swimmer 96x48x48 (4000 steps)", 400, 100, 4000))


def cpu_scenarios(args):
    from paper_1108_0786_gb300 import workloads as wl
    return (wl.three_sphere_periodic(), wl.channel_swimmer(), workload(args, 0), wl.design_swimmer())


def cpu_baseline(args, full=False):
    """The FP64 oracle, as it stands, on the host cores: each config timed at
    all threads and at one thread, after one untimed step, over a bounded
    sample of its steps (every step with ``full``).  The headline value is
    the benchmark's own workload at all threads."""
    import oracle
    threads = oracle.num_threads()
    out = {}
    for (name, n_all, n_one, n_full), sc in zip(CPU_SAMPLES, cpu_scenarios(args)):
        name = name.format(nx=sc.nx, ny=sc.ny, nz=sc.nz)
        row = {"cells": sc.cells, "full_steps": n_full}
        for label, nt, n in (("all_threads", threads, n_all), ("one_thread", 1, n_one)):
            n = n_full if full else n
            oracle.set_num_threads(nt)
            o = oracle.from_scenario(sc)
            o.step(1)
            t0 = time.perf_counter()
            o.step(n)
            dt = time.perf_counter() - t0
            o.close()
            row[label] = {"mlups": round(sc.cells * n / dt / 1e6, 2), "threads": nt, "steps": n,
                          "seconds": round(dt, 2)}
        out[name] = row
    oracle.set_num_threads(threads)
    sc = cpu_scenarios(args)[2]
    head = out[CPU_SAMPLES[2][0].format(nx=sc.nx, ny=sc.ny, nz=sc.nz)]["all_threads"]
    return {"value": head["mlups"], "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{head['steps']} coupled FP64 steps of the full {sc.nx}x{sc.ny}x{sc.nz} workload "
                      f"({len(sc.bodies)} capsules) after 1 untimed step, {threads} threads; every config below "
                      f"at {threads} threads and at 1 thread, steps run as listed",
            "configs": out}


# ---- arms ------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import torch
    from paper_1108_0786_gb300 import _build, lbm
    if rank == 0 or world > 1:
        _build.build()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    sc = workload(args, rank)
    lat = lbm.from_scenario(sc, precision=args.precision,
                            options=lbm.OPT_OVERLAP if args.overlap else 0)
    if args.shape != "auto":
        shape = tuple(int(v) for v in args.shape.split(","))
        lat.tune(*shape)               # a fixed bulk-kernel shape must be set before the first step
    lat.step(1)
    if args.shape == "auto":
        shape = lat.autotune(5)        # the library's autotuner picks the bulk-kernel shape
    lat.step(args.warmup)
    lat.sync()
    with ClockSampler(local) as clk:
        ms = timed_steps(lat, args.steps, world, device)
    clocks = clk.summary()
    value = job_mlups(sc.cells, args.steps, world, ms)
    # dominant kernel: per-launch durations with CUDA events on the launching stream
    kms = lat.time_kernels(50)
    bpc = lat.bytes_per_cell
    peak, peak_kind = hbm_peak()
    achieved = bpc * sc.cells / (kms["stream_collide"] / 1e3) / 1e9
    traffic = recorded_traffic(sc.cells)
    launches = lat.kernels_per_step * args.steps
    lat.close()
    torch.cuda.empty_cache()
    e2e = e2e_run(sc, args, world, device)
    torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16", "bf16": "bf16", "f64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"capsule swarm {sc.nx}x{sc.ny}x{sc.nz} periodic D3Q19, tau=1, "
                               f"8 three-capsule swimmers (r=4, l=8), {args.precision} deviation storage",
                   "cells": sc.cells, "bodies": len(sc.bodies), "springs": len(sc.springs),
                   "bulk_kernel_shape": {"cells_per_thread": shape[0], "min_blocks_per_sm": shape[1]},
                   "precision": args.precision, "replicas": world,
                   "l2": "inputs larger than L2: %.2f GB of populations per step vs 129 MB L2"
                         % (bpc * sc.cells / 1e9)},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "stream_collide", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": None if traffic is None else round(traffic),
                     "algorithmic_bytes": bpc * sc.cells,
                     "launch_ms": round(kms["stream_collide"], 4),
                     "per_kernel_ms": {k: round(v, 4) for k, v in kms.items()}},
        "clocks": clocks,
    }
    if not args.no_variants and rank == 0 and world == 1:
        ens = ensemble_run()
        # the oracle runs of the ensemble's members proceed on the host cores
        # (one left to the launching thread) during the GPU-bound parts below
        pool, pending = start_oracle_members()
        line["storage_variants"] = variant_runs(workload(args, 0), 2000)
        line["adjoint"] = adjoint_run()
        line["ensemble"] = ensemble_errors(ens, pending.get())
        pool.close()
        pool.join()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)


def adjoint_run(precision="f32", segment=64):
    """Reverse sweep against the forward run on the 96 x 48 x 48 gradient
    study (one three-sphere swimmer, 4000 steps): wall-clock of the forward
    steps alone, of the recorded forward (lbm_adjoint_record) and of the
    reverse sweep (lbm_adjoint_backward: recomputation from checkpoints every
    `segment` steps plus the transposed steps), each bracketed by a device
    synchronisation."""
    import numpy as np
    from paper_1108_0786_gb300 import lbm, workloads as wl
    sc = wl.design_swimmer(capsules=False)
    seed = np.zeros((len(sc.bodies), 13))
    seed[1, 0] = 1.0                    # x of the middle body: its displacement
    times = {}
    lat = lbm.from_scenario(sc, precision=precision)
    lat.step(64)
    lat.sync()
    t0 = time.perf_counter()
    lat.step(sc.steps)
    lat.sync()
    times["forward"] = time.perf_counter() - t0
    lat.close()
    lat = lbm.from_scenario(sc, precision=precision)
    lat.step(0)                                 # device buffers and step graphs
    lat.sync()
    t0 = time.perf_counter()
    lat.adjoint_record(sc.steps, segment)
    times["record"] = time.perf_counter() - t0
    lat.adjoint_backward(seed)                  # warm-up of the reverse kernels
    t0 = time.perf_counter()
    g = lat.adjoint_backward(seed)
    times["backward"] = time.perf_counter() - t0
    lat.close()
    signs = np.sign([d.amp for d in sc.drives])
    return {"workload": f"{sc.name}, {sc.steps} steps, {precision} storage, checkpoints every {segment} steps",
            "forward_ms": round(times["forward"] * 1e3, 2), "record_ms": round(times["record"] * 1e3, 2),
            "backward_ms": round(times["backward"] * 1e3, 2),
            "backward_over_forward": round(times["backward"] / times["forward"], 3),
            "record_plus_backward_over_forward": round((times["record"] + times["backward"]) / times["forward"], 3),
            "d_displacement_d_amplitude": float((g["drive"][:, 0] * signs).sum()),
            "d_displacement_d_k": float(g["spring"][:, 0].sum())}


def _oracle_member_run(index):
    """(start, final) body positions of ensemble member `index` run by the
    FP64 oracle for its full step count (one process, one thread)."""
    import oracle
    from paper_1108_0786_gb300 import workloads as wl
    oracle.set_num_threads(1)
    sc = wl.ensemble_members()[index]
    o = oracle.from_scenario(sc)
    x0 = o.bodies()[:, 0:3].copy()
    o.step(sc.steps)
    return index, x0, o.bodies()[:, 0:3].copy()


def start_oracle_members(edge=48):
    """The oracle runs of every ensemble member of the given edge, started on
    a pool of spawned processes (they share no CUDA state); returns the pool
    and the pending results."""
    import multiprocessing as mp
    from paper_1108_0786_gb300 import workloads as wl
    idx = [i for i, sc in enumerate(wl.ensemble_members()) if sc.nx == edge]
    pool = mp.get_context("spawn").Pool(processes=max(1, min(len(idx), (os.cpu_count() or 2) - 1)))
    return pool, pool.map_async(_oracle_member_run, idx)


def ensemble_run(precision="f32", reference_edge=48):
    """The 96-box ensemble (one swimmer per periodic box, edges 48-96, 1000 /
    2000 / 4000 steps) in batched mode: one launch of each per-step kernel
    over each half of the members, the bulk shape chosen by the ensemble
    autotuner; then
    the whole ensemble runs to completion; aggregate MLUPS = sum of cells x
    steps over the wall-clock between two device synchronisations.  Member
    error: every member of edge `reference_edge` against the FP64 oracle at
    its full step count (run on spawned processes meanwhile), the relative
    error of each body's displacement."""
    import numpy as np
    from paper_1108_0786_gb300 import lbm, workloads as wl
    scs = wl.ensemble_members()
    lats = [lbm.from_scenario(sc, precision=precision) for sc in scs]
    x0 = [lat.bodies()[:, 0:3].copy() for lat in lats]
    ens = lbm.Ensemble(lats)
    ens.step([16] * len(lats))                  # builds the graphs; members then restart their count
    vec = ens.autotune(3)
    ens.step([16] * len(lats))
    ens.sync()
    steps = [sc.steps - 32 for sc in scs]
    t0 = time.perf_counter()
    ens.step(steps)
    ens.sync()
    dt = time.perf_counter() - t0
    updates = sum(sc.cells * n for sc, n in zip(scs, steps))
    final = [lat.bodies() for lat in lats]
    # per step and storage type: 8 kernels in each of the two chains (halves of the members)
    launches = 8 * 16 * 2 * len({lat.precision for lat in lats})
    ens.close()
    for lat in lats:
        lat.close()
    return {"workload": f"{len(scs)} periodic boxes (edges 48-96, {sum(sc.cells for sc in scs) / 1e6:.1f} M cells), "
                        f"one three-body swimmer each, 1000/2000/4000 steps, {precision} storage",
            "mode": "batched: per step one launch of each per-step kernel over each half of the members "
                    "(two chains, latency-bound kernels at high stream priority beside the other half's bulk kernel)",
            "mlups": round(updates / dt / 1e6, 1), "wall_s": round(dt, 3), "cell_updates": updates,
            "bulk_cells_per_thread": vec, "launches_per_16_steps": launches,
            "_final": final, "_x0": x0, "_edge": reference_edge}


def ensemble_errors(res, results):
    """Per-member displacement error of the GPU ensemble against the oracle."""
    import numpy as np
    errors = []
    for i, ox0, oxb in results:
        d_ref = np.linalg.norm(oxb - ox0, axis=1)
        d = np.linalg.norm(res["_final"][i][:, 0:3] - res["_x0"][i], axis=1)
        errors.append(float(np.abs(d - d_ref).max() / d_ref.max()))
    for k in ("_final", "_x0", "_edge"):
        res.pop(k, None)
    res["member_displacement_rel_err_vs_oracle"] = {
        "members": len(errors), "edge": 48, "steps": "full (1000/2000/4000)",
        "max": max(errors) if errors else None, "median": float(np.median(errors)) if errors else None}
    return res


REFERENCE_BUDGET_S = 90.0


def run_reference(args, world, rank):
    """The oracle as the reference arm, on the benchmark's own workload (the
    full 512 x 256 x 256 capsule swarm, FP64, all host cores).  Warm-up is
    at most 2 steps; the timed steps are the requested count, bounded so
    that they take about REFERENCE_BUDGET_S seconds (one oracle step of this
    workload takes ~0.5 s on 16 cores), and the line reports the count run."""
    if rank != 0:
        return
    import oracle
    sc = workload(args, 0)
    o = oracle.from_scenario(sc)
    warm = max(1, min(args.warmup, 2))
    t0 = time.perf_counter()
    o.step(warm)
    per_step = (time.perf_counter() - t0) / warm
    n = max(1, min(args.steps, int(REFERENCE_BUDGET_S / per_step)))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    o.close()
    value = sc.cells * n / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT,
            "n_gpus": world, "steps": n, "steps_requested": args.steps, "warmup": warm,
            "ms_per_step": round(dt * 1e3 / n, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"capsule swarm {sc.nx}x{sc.ny}x{sc.nz} periodic D3Q19, tau=1, "
                                   f"8 three-capsule swimmers (r=4, l=8), FP64 CPU oracle",
                       "cells": sc.cells, "bodies": len(sc.bodies), "springs": len(sc.springs)},
            "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{n} coupled FP64 steps of the benchmark's workload after {warm} "
                                       f"untimed, bounded to ~{REFERENCE_BUDGET_S:.0f} s"},
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.cpu_only:
        if rank == 0:
            print(json.dumps({"cpu_baseline": cpu_baseline(args, full=args.cpu_full)}), flush=True)
    elif args.only:
        if rank == 0:
            from paper_1108_0786_gb300 import _build
            _build.build()
            if args.only == "ensemble":
                r = ensemble_run()
                for k in ("_final", "_x0", "_edge"):
                    r.pop(k, None)
            else:
                r = adjoint_run()
            print(json.dumps({args.only: r}), flush=True)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
