"""Benchmark of the damped-current PML PIC step on GB300.

Default workload (the N=1 line; one step = one PIC time step over the whole
particle set, i.e. all hot-path stages: sort every 20 steps, gather + Boris
push + move + Esirkepov deposit + alpha-damped flush, split-field PML Yee
update of E and B):
  3D plasma + drifting beam: 256 x 256 x 512 physical cells of 1 um + a
  16-cell damped-current PML on every face (288 x 288 x 544 cells), electrons
  and protons 8 per cell each (536,870,912 macroparticles, drawn on the
  device from a seeded generator), Maxwellian u_th = 0.01, plus an electron
  beam at u_z = 5 (41,177 particles, neutralised by immobile ions) heading
  into the +z PML; order 1, dt = 0.99 x Courant limit, FP32 fields and
  momenta with IEEE FP64 PML split parts.  The autotuner picks the launch
  shapes (the tile-resident particle kernel for this plasma).
Metric: particle-steps/s (live particles pushed per second, counted on the
device); cell-updates/s of the Yee/PML update beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line with "roofline" (the particle kernel's algorithmic
bytes per launch over its CUDA-event time, against the measured copy
bandwidth), "e2e" (the same steps through the C ABI with the particle
records uploaded from pinned host memory inside the timed region and each
step's particle-step count read back), "float_float_parts" (the same run with
float-float PML parts), "beam_3d" (the 128^3 + 16 beam of 4,194,304
particles), "batch2d" (4096 batched 2D runs, FP32 and FP64) and
"cpu_baseline" (the FP64 oracle on the plasma + beam workload reduced to
24 x 24 x 48 + 8 cells, with the GPU's max relative field error on that
sample).  --impl reference times the oracle alone on that sample.
--beam, --plasma, --single-particle, --cavity and --precision-study measure
the other workloads (their own JSON lines).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NPHYS = (128, 128, 128)
PML = (16,) * 6
D = (1e-6, 1e-6, 1e-6)
NPART = 4_194_304
SORT_EVERY = 20
METRIC = "particle-steps/s"


def beam_center():
    return (PML[0] + NPHYS[0] / 2 + 0.3, PML[2] + NPHYS[1] / 2 + 0.1, PML[4] + NPHYS[2] - 24 + 0.2)


def workload(order, theta, prec, npart=NPART):
    return {"workload": f"3D beam exiting +z PML: {NPHYS[0]}^3 + {PML[0]}-cell PML, {npart} macroparticles, "
                        f"order {order}, theta {theta} deg, {prec} fields + fp64 PML splits",
            "grid": [n + 2 * p for n, p in zip(NPHYS, PML[::2])], "particles": npart,
            "shape_order": order, "theta_deg": theta, "alpha": "damped (Eq. alpha, v=c)",
            "sort_every": SORT_EVERY, "l2": "working set > L2 (particles 134 MB + fields ~550 MB)",
            "data": "synthetic"}


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(n_live, occ_cells, n_int, n_pml, prec, bn=False):
    """Algorithmic bytes of one step: each operand read once, each result
    written once.  Particle (3D FP32): 32 B read + 28 B written; occupied cell
    gather/deposit: 9 field words read (E and both B half steps) + 3 current
    words written (48 B; 96 B in FP64), or, with bn (the tile kernel, which
    reads B at the integer time written by the field step), 6 field words
    read + 3 written (36 B).  Yee interior cell: E, B, J read, E, B written
    (60 B FP32, 120 B FP64); PML cell: 12 FP64 split parts read+written, J
    read, E, B written (228 B; 252 B FP64); with bn the B pass also writes B
    at the integer time (+12 B per cell)."""
    e = 8 if prec == "fp64" else 4
    words = 9 if bn else 12
    part = (60 if prec != "fp64" else 104) * n_live + words * e * occ_cells
    field = (15 * e) * n_int + (192 + 9 * e) * n_pml + (12 * (n_int + n_pml) if bn else 0)
    return part, field


def count_cells():
    N = [n + 2 * p for n, p in zip(NPHYS, PML[::2])]
    total = N[0] * N[1] * N[2]
    interior = NPHYS[0] * NPHYS[1] * NPHYS[2]
    return total, interior, total - interior


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu
# capture of the full workload) of the fused order-1 kernel with 4 particles
# per thread, FP32, theta 0; keyed by (order, particles per thread, prec,
# theta, particles).  Reset to {} whenever that kernel changes.  Captured with
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:k_pd1 -s 3 -c 1
#       python bench.py --beam --tuning 4,1 --steps 3 --warmup 3 --no-cpu-baseline --no-batch --no-fp64
# (the first timed step: 138,749,696 B read + 78,776,320 B written).
NCU_TRAFFIC = {(1, 4, "fp32", 0.0, 4194304): 138_749_696 + 78_776_320}


def combine_ranks(ms, psteps, ms_e2e, ps_e2e, world, device):
    """Whole-job figures of N replicas: the slowest rank's times (max over
    ranks) and the particle-steps of all ranks (sum)."""
    if world == 1:
        return ms, psteps, ms_e2e, ps_e2e
    import torch
    vals = torch.tensor([ms, psteps, ms_e2e, ps_e2e], dtype=torch.float64, device=device)
    mx = vals.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = vals.clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(mx[2]), float(sm[3])


def run_gpu(args, rank, world):
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Sim, pack_particles
    from paper_2201_09084_gb300 import build as B

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        torch.distributed.barrier()
    npart = args.particles
    parts = I.beam(3, npart, NPHYS, PML, beam_center(), theta_deg=args.theta)[0]
    stream = torch.cuda.current_stream()
    sim = Sim(3, NPHYS, D, PML, cfl=0.99, order=args.order, prec=args.prec, alpha_mode="damped",
              sort_every=0, split_fp64=True, stream=stream)
    pos, mom = pack_particles(parts["cell"], parts["off"], parts["u"], parts["w"], args.prec)
    sim.add_species(pos, mom, npart, parts["q"], parts["m"])
    pos0, mom0 = pos.clone(), mom.clone()
    sim.sort()
    if args.tuning:
        p_, k_ = (int(x) for x in args.tuning.split(","))
        sim.set_tuning(p_, k_)
        tuning = {"particles_per_thread": p_, "z_nodes_per_thread": k_, "source": "--tuning"}
    else:
        tuning = sim.autotune(steps=3)   # launch shapes, from a restored snapshot

    def one_step(i, ev=None):
        if i % SORT_EVERY == 0:
            sim.sort()
        if ev is not None:
            ev[0].record(stream)
        sim.push_deposit()
        if ev is not None:
            ev[1].record(stream)
        sim.field_step()
        if ev is not None:
            ev[2].record(stream)

    for i in range(args.warmup):
        one_step(i)
    sim.sync()
    ps0 = sim.particle_steps()
    l0 = sim.launch_count()
    # occupied cells at the start of the timed region (for the byte model)
    cells = mom.view(torch.int32)[:, 3]
    occ = int(torch.unique(cells[cells >= 0]).numel())
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for i in range(args.steps):
        one_step(args.warmup + i, evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    sim.sync()
    ms = t0.elapsed_time(t1)
    psteps = sim.particle_steps() - ps0
    launches = sim.launch_count() - l0
    t_pd = np.mean([e[0].elapsed_time(e[1]) for e in evs])
    t_f = np.mean([e[1].elapsed_time(e[2]) for e in evs])

    # ---- end to end through the public API from pinned host buffers ----
    hpos = pos0.cpu().pin_memory()
    hmom = mom0.cpu().pin_memory()
    sim2 = Sim(3, NPHYS, D, PML, cfl=0.99, order=args.order, prec=args.prec, alpha_mode="damped",
               sort_every=SORT_EVERY, stream=stream)
    sim2.set_tuning(tuning["particles_per_thread"], tuning["z_nodes_per_thread"])
    dpos = torch.empty_like(pos0)
    dmom = torch.empty_like(mom0)
    sim2.add_species(dpos, dmom, npart, parts["q"], parts["m"])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nsteps_e2e = args.warmup + args.steps
    e0.record(stream)
    dpos.copy_(hpos, non_blocking=True)
    dmom.copy_(hmom, non_blocking=True)
    for _ in range(nsteps_e2e):
        sim2.step(1)
        ps_e2e = sim2.particle_steps()   # each step's result read back (synchronising 8-byte copy)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)

    # ---- reductions over ranks ----
    ms, psteps, ms_e2e, ps_e2e = combine_ranks(ms, psteps, ms_e2e, ps_e2e, world, "cuda")
    value = psteps / (ms / 1e3)
    total_cells, n_int, n_pml = count_cells()
    cell_updates = world * total_cells * args.steps / (ms / 1e3)
    n_live_avg = (psteps / world) / args.steps
    b_part, b_field = algorithmic_bytes(n_live_avg, occ, n_int, n_pml, args.prec)
    peak, peak_kind = measured_peak()
    traffic = None
    if t_pd >= t_f:
        name = ("k_pd1 (fused order-1 gather/push/move/deposit/damp)" if args.order == 1
                else "k_particles (fused gather/push/move/deposit/damp)")
        dom, t_dom, b_dom = name, t_pd, b_part
        traffic = NCU_TRAFFIC.get((args.order, tuning["particles_per_thread"], args.prec, args.theta, npart))
    else:
        dom, t_dom, b_dom = "field_step (k_field_E + k_field_B)", t_f, b_field
    achieved = b_dom / (t_dom / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "f64",
        "data": "synthetic",
        "config": dict(workload(args.order, args.theta, args.prec, npart), parallelism=f"replicas x{world}"),
        "cell_updates_per_s": cell_updates,
        "kernel_ms": {"push_deposit": t_pd, "field_step": t_f},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} (copy)", "traffic": traffic,
                     "algorithmic_bytes_per_launch": b_dom},
        "e2e": {"value": ps_e2e / (ms_e2e / 1e3), "unit": "particle-steps/s",
                "h2d_bytes_per_step": 2 * npart * (32 if args.prec == "fp64" else 16) / nsteps_e2e,
                "d2h_bytes_per_step": 8,
                "note": f"pinned host particles copied in once per run of {nsteps_e2e} steps (h2d bytes "
                        "are that copy per step); every step runs step_n (sorting every 20 steps) and "
                        "reads its particle-step count back to the host"},
        "gpu_launches": int(launches),
        "autotune": tuning,
        "clocks": clk,
    }
    return out


# ----------------------------------------------------------------------------
def run_batch(steps, warmup, prec, nruns=4096, order=3):
    """Batched independent 2D runs: nruns single-particle boxes with sizes
    U{64..256} x U{64..256}, PML U{8..24} cells, angle U[0, 80] deg from +z,
    gamma log-uniform in [1.1, 100]; one persistent launch per step replayed
    from a CUDA graph.  Returns a dict of rates and the roofline of the step
    kernel (algorithmic bytes: 60 B per interior cell, 164 B per PML cell in
    FP32 (8 split parts read and written); 120 / 248 B in FP64)."""
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Batch, pack_particles
    r = I.batched_runs(nruns)
    pos, mom = pack_particles(r["cell"], r["off"], r["u"], r["w"], prec)
    b = Batch(r["nx"], r["nz"], r["npml"], (D[0], D[2]), pos, mom, r["q"], r["m"], cfl=0.99, order=order,
              prec=prec, alpha_mode="damped")
    stream = torch.cuda.current_stream()
    b.step(warmup)
    b.sync()
    p0 = b.particle_steps()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ps = b.particle_steps() - p0
    nx, nz, npml = r["nx"].astype(np.int64), r["nz"].astype(np.int64), r["npml"].astype(np.int64)
    cells = int(np.sum((nx + 2 * npml) * (nz + 2 * npml)))
    interior = int(np.sum(nx * nz))
    e = 8 if prec == "fp64" else 4
    byts = 15 * e * interior + (128 + 9 * e) * (cells - interior)
    peak, kind = measured_peak()
    achieved = byts / (ms / steps / 1e3) / 1e9
    tuning = b.tuning()
    b.close()
    return {"workload": f"{nruns} independent 2D runs, 64-256 cells per side, PML 8-24, one electron each, "
                        f"angle 0-80 deg, gamma 1.1-100, order {order}, {prec}",
            "steps": steps, "ms_per_step": ms / steps, "cell_updates_per_s": cells * steps / (ms / 1e3),
            "particle_steps_per_s": ps / (ms / 1e3), "cells": cells, "autotune": tuning,
            "roofline": {"bound": "hbm", "kernel": "k_batch_step", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{kind} (copy)",
                         "algorithmic_bytes_per_launch": byts},
            "launches_per_step": 1, "graph": "two steps per captured graph"}


def cpu_sample(order, theta, sample, steps):
    """The oracle on a bounded sample of the workload: the full 160^3 grid,
    `sample` beam particles (weights scaled to the same charge), `steps` time
    steps.  Returns (particle-steps/s scaled to the full particle count,
    description).  The particle stages are timed separately from the field
    update so the full-workload rate is t_field + N t_particle per step."""
    import oracle as O
    from paper_2201_09084_gb300 import inputs as I
    oracle_build = O.build()
    dt = O.yee_dt(D, 0.99, 3)
    parts = I.beam(3, sample, NPHYS, PML, beam_center(), theta_deg=theta)[0]
    sim = O.OracleSim(3, NPHYS, PML, D, dt, order=order, alpha_mode="damped")
    X = I.absolute(parts["cell"], parts["off"])
    u = parts["u"].astype(np.float64)
    sim.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2],
                      parts["w"].astype(np.float64) * (NPART / sample), parts["q"], parts["m"])
    t_part = t_field = 0.0
    for _ in range(steps):
        a = time.perf_counter()
        sim.push()
        sim.deposit()
        b = time.perf_counter()
        sim.field_E()
        sim.field_B()
        c = time.perf_counter()
        t_part += b - a
        t_field += c - b
    per_particle = t_part / steps / sample
    step_full = t_field / steps + per_particle * NPART
    value = NPART / step_full
    desc = (f"FP64 C oracle, 1 thread: {steps} steps of the full 160^3 grid with a {sample}-particle "
            f"sample of the beam; rate = N / (t_field + N t_particle), N = {NPART}")
    return value, desc, step_full


def cpu_batch_sample(nruns=4096, sample=64, steps=20, order=3):
    """The oracle on a bounded sample of the batched 2D runs: the first
    `sample` of the same `nruns` runs (their sizes, PML widths, angles and
    Lorentz factors), one FP64 box each, `steps` steps, one after another on
    one core.  The time per cell-step of the sample scales to the whole batch
    by its cell count.  Returns (particle-steps/s, cell-updates/s,
    description)."""
    import oracle as O
    from paper_2201_09084_gb300 import inputs as I
    O.build()
    r = I.batched_runs(nruns)
    dt = O.yee_dt(D, 0.99, 2)
    nx, nz, npml = r["nx"].astype(np.int64), r["nz"].astype(np.int64), r["npml"].astype(np.int64)
    cells_all = int(np.sum((nx + 2 * npml) * (nz + 2 * npml)))
    t = 0.0
    cells_sample = 0
    sample = min(sample, nruns)
    for k in range(sample):
        p = int(npml[k])
        sim = O.OracleSim(2, (int(nx[k]), 0, int(nz[k])), (p, p, 0, 0, p, p), D, dt, order=order,
                          alpha_mode="damped")
        X = I.absolute(r["cell"][k:k + 1], r["off"][k:k + 1])
        u = r["u"][k].astype(np.float64)
        sim.add_particles(X[:, 0], X[:, 1], X[:, 2], [u[0]], [u[1]], [u[2]], [1.0], r["q"], r["m"])
        a = time.perf_counter()
        sim.step(steps)
        t += time.perf_counter() - a
        cells_sample += (int(nx[k]) + 2 * p) * (int(nz[k]) + 2 * p)
    per_cell_step = t / (steps * cells_sample)
    step_all = per_cell_step * cells_all
    desc = (f"FP64 C oracle, 1 thread: the first {sample} of the {nruns} runs, {steps} steps each, "
            f"scaled by cells ({cells_sample} of {cells_all})")
    return nruns / step_all, cells_all / step_all, desc


SP_NPHYS = (128, 0, 128)
SP_PML = (16, 16, 0, 0, 16, 16)
SP_GAMMA = float(np.sqrt(101.0))


def single_particle_bytes():
    """Algorithmic bytes of one FP64 field step of the 2D single-particle box:
    interior cell E, B, J read and E, B written (120 B); PML cell 8 FP64 split
    parts read and written plus J read and E, B written (200 B)."""
    nint = SP_NPHYS[0] * SP_NPHYS[2]
    total = (SP_NPHYS[0] + SP_PML[0] + SP_PML[1]) * (SP_NPHYS[2] + SP_PML[4] + SP_PML[5])
    return 120 * nint + 200 * (total - nint), total


def cpu_single_particle(steps):
    """The oracle on the whole 2D single-particle workload (it is small
    enough to run in full): 128 x 128 cells + 16-cell PML, an electron with
    u_z = 10 and its motionless partner, order 1, damped PML, `steps` steps on
    one core.  Returns (particle-steps/s, cell-updates/s, description)."""
    import oracle as O
    from paper_2201_09084_gb300 import inputs as I
    O.build()
    dt = O.yee_dt(D, 0.99, 2)
    sim = O.OracleSim(2, SP_NPHYS, SP_PML, D, dt, order=1, alpha_mode="damped")
    for sp in I.single_pair(2, SP_NPHYS, SP_PML, gamma=SP_GAMMA):
        X = I.absolute(sp["cell"], sp["off"])
        u = sp["u"].astype(np.float64)
        sim.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], sp["w"].astype(np.float64),
                          sp["q"], sp["m"], sp["immobile"])
    t, psteps = 0.0, 0
    for _ in range(steps):
        psteps += int(sim.particles()["alive"][0])   # the mover, before this step's push
        a = time.perf_counter()
        sim.step(1)
        t += time.perf_counter() - a
    _, total = single_particle_bytes()
    desc = f"FP64 C oracle, 1 thread: the whole workload, {steps} steps"
    return psteps / t, total * steps / t, desc


def run_single_particle(args):
    """The 2D FP64 single-particle workload of the paper's studies: 128 x 128
    cells of 1 um + 16-cell PML on all sides, an electron with u_z = 10
    (gamma = sqrt(101)) and its motionless partner at the centre moving into
    the +z PML, order 1, damped PML, dt = 0.99 x the Courant limit.  W
    untimed steps on a throw-away box, then `steps` steps of a fresh box from
    t = 0 (the workload is 400 steps) through step_n, timed with CUDA events.
    The step is one field update of 25,600 cells and a push of at most one
    particle: launch- and latency-bound.  Prints its own JSON line."""
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Sim, pack_particles
    from paper_2201_09084_gb300 import build as B
    B.build()
    stream = torch.cuda.current_stream()

    def make():
        sim = Sim(2, SP_NPHYS, D, SP_PML, cfl=0.99, order=1, prec="fp64", alpha_mode="damped", sort_every=0,
                  stream=stream)
        keep = []
        for sp in I.single_pair(2, SP_NPHYS, SP_PML, gamma=SP_GAMMA):
            pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp64")
            sim.add_species(pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"])
            keep.append((pos, mom))
        return sim, keep

    warm, keep_w = make()
    warm.step(args.warmup)
    warm.sync()
    sim, keep = make()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    l0 = sim.launch_count()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    psteps = sim.particle_steps()
    launches = sim.launch_count() - l0
    byts, total = single_particle_bytes()
    peak, kind = measured_peak()
    achieved = byts / (ms / args.steps / 1e3) / 1e9
    out = {"metric": METRIC, "value": psteps / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "2D single particle: 128x128 + 16-cell PML, electron u_z 10 + partner, "
                                  "order 1, fp64, damped PML", "cells": total},
           "cell_updates_per_s": total * args.steps / (ms / 1e3),
           "roofline": {"bound": "hbm", "kernel": "whole step (field update + push)", "achieved": achieved,
                        "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{kind} (copy)",
                        "traffic": None, "algorithmic_bytes_per_step": byts,
                        "note": "3.8 MB per step fits in L2; the step is launch- and latency-bound"},
           "gpu_launches": int(launches), "clocks": clk}
    if not args.no_cpu_baseline:
        v, cu, desc = cpu_single_particle(args.steps)
        out["cpu_baseline"] = {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                               "sample": desc, "cell_updates_per_s": cu}
    sim.close()
    warm.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    sample = max(16384, int(262144 / max(1, (args.steps + args.warmup) / 20)))
    v, desc, step_full = cpu_sample(args.order, args.theta, sample, args.steps + args.warmup)
    out = {"metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_full * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": dict(workload(args.order, args.theta, "fp64"), parallelism="cpu oracle"),
           "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return out


def run_precision_study(args):
    """Precision study on the plasma + beam workload (128 x 128 x 256 cells +
    16-cell PML, electrons and protons 8 per cell, Maxwellian u_th = 0.01,
    drifting beam at u_z = 5, order 1, sort every 20 steps): the FP32 forms
    (float-float PML parts, IEEE FP64 parts, int64 deterministic deposition)
    against the plain FP64 form on the GPU at full size, with each form's
    throughput; and every form against the FP64 CPU oracle on the same
    workload reduced to 24 x 24 x 48 + 8 cells for 20 steps (the plasma is
    chaotic, so forms separate physically after a few tens of steps)."""
    import torch
    import oracle as O
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Sim, pack_particles
    from paper_2201_09084_gb300 import build as B
    B.build()
    names = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
    forms = [("fp64", "fp64", False), ("fp32", "fp32", False), ("fp32-splitfp64", "fp32", True),
             ("fixed64", "fixed64", False)]

    def run(nphys, pml, parts, prec, split, steps, marks, dt):
        sim = Sim(3, nphys, D, pml, dt=dt, order=1, prec=prec, alpha_mode="damped", sort_every=20,
                  split_fp64=split)
        keep = []
        for sp in parts:
            pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], prec)
            sim.add_species(pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"])
            keep.append((pos, mom))
        sim.sort()
        sim.autotune(steps=3)   # launch shapes from a restored snapshot (a thermal plasma: one thread per particle)
        snaps, done, t = {}, 0, 0.0
        for m in marks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sim.step(m - done)
            e1.record()
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1)
            done = m
            snaps[m] = {k: sim.field(k).cpu().numpy() for k in names}
            dg = sim.diag()
            snaps[m]["gauss"] = dg["gauss"] / dg["rho_scale"] if dg["rho_scale"] > 0 else None
        ps = sim.particle_steps()
        sim.close()
        del keep
        torch.cuda.empty_cache()
        return snaps, ps / (t / 1e3)

    def err(a, b):
        scale = max(max(np.abs(b[k]).max() * (C if k[0] == "B" else 1.0) for k in names), 1e-300)
        return max(np.abs(a[k] - b[k]).max() * (C if k[0] == "B" else 1.0) for k in names) / scale

    C = 299792458.0
    out = {"metric": "max relative field error vs FP64", "unit": "1", "higher_is_better": False,
           "data": "synthetic", "config": {"workload": "precision study: plasma + drifting beam, "
                                            "128x128x256 + 16-cell PML, 8 ppc e- and p+, u_th 0.01, "
                                            "beam u_z 5, order 1"}}
    # full size, GPU forms against the GPU FP64 form
    nphys, pml = (128, 128, 256), (16,) * 6
    parts = I.plasma(nphys, pml, D[0])
    dt = None
    import oracle as _O
    dt = _O.yee_dt(D, 0.99, 3)
    marks = (20, args.steps if args.steps > 20 else 50)
    res = {}
    ref = None
    for label, prec, split in forms:
        snaps, rate = run(nphys, pml, parts, prec, split, marks[-1], marks, dt)
        if label == "fp64":
            ref = snaps
        res[label] = {"particle_steps_per_s": rate,
                      "gauss_rel": {str(m): snaps[m]["gauss"] for m in marks},
                      "err_vs_fp64": {str(m): (err(snaps[m], ref[m]) if ref is not None else 0.0) for m in marks}}
    out["full_size"] = {"steps": list(marks), "particles": int(sum(len(p["w"]) for p in parts)), "forms": res}
    # reduced size, every form against the oracle
    nphys_s, pml_s = (24, 24, 48), (8,) * 6
    parts_s = I.plasma(nphys_s, pml_s, D[0], beam_radius=4.0, beam_length=12.0)
    ora = O.OracleSim(3, nphys_s, pml_s, D, dt, order=1, alpha_mode="damped")
    for sp in parts_s:
        X = I.absolute(sp["cell"], sp["off"])
        u = sp["u"].astype(np.float64)
        ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], sp["w"].astype(np.float64),
                          sp["q"], sp["m"], sp["immobile"])
    oref = {}
    for m in (10, 20):
        ora.step(10)
        oref[m] = {k: ora.field(k) for k in names}
    small = {}
    for label, prec, split in forms:
        snaps, _ = run(nphys_s, pml_s, parts_s, prec, split, 20, (10, 20), dt)
        small[label] = {"err_vs_oracle": {str(m): err(snaps[m], oref[m]) for m in (10, 20)},
                        "gauss_rel": {str(m): snaps[m]["gauss"] for m in (10, 20)}}
    out["vs_oracle_reduced"] = {"grid": "24x24x48 + 8-cell PML", "steps": [10, 20], "forms": small}
    out["value"] = small["fp32"]["err_vs_oracle"]["20"]
    return out

# DRAM bytes per particle-step of the one-thread-per-particle kernel on the
# thermal plasma (dram__bytes_read.sum + dram__bytes_write.sum of the three
# launches of one step, electrons + protons + beam, 557,966,080 B for
# 8,429,785 particles), from one ncu capture of the 64 x 64 x 128 case with
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,... --clock-control none
#       -k regex:k_particles -s 9 -c 3
#       python bench.py --plasma --plasma-cells 64,64,128 --tuning 1,1 --steps 3 --warmup 3
# The plasma fills the box at a fixed 8 particles per cell, so the traffic
# grows with the particle count; the full-size figure is scaled by it.  Set
# to None whenever that kernel changes.
PLASMA_NCU_BYTES_PER_PARTICLE = 557_966_080 / 8_429_785

# DRAM bytes per particle-step of the tile kernel on the plasma (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch over the particles it pushed), from an ncu
# capture of the 64 x 64 x 128 case; the plasma fills the box at a fixed 8 particles
# per cell and species, so the traffic grows with the particle count and the
# full-size figure is scaled by it.  None until captured on the current kernel.
# Captured with
#   ncu --set full --clock-control none -k regex:^k_tile$ -s 4 -c 1
#       python bench.py --cells 64,64,128 --no-extra --no-cpu-baseline --steps 3 --warmup 3 --tuning 2,1
# (308,050,176 B read + 223,579,392 B written for 8,429,785 particles).
HEADLINE_NCU_BYTES_PER_PARTICLE = (308_050_176 + 223_579_392) / 8_429_785
HEADLINE_NCU_NOTE = ("per launch: dram__bytes_read.sum + dram__bytes_write.sum of the tile kernel on the "
                     "64x64x128 case (63.1 B per particle), scaled by the particles pushed")

# Plasma boxes with more particles per species than this are generated and
# packed one z-plane of cells at a time (inputs.plasma_planes) instead of in
# one piece, so host memory holds one plane.
STREAM_PARTICLES = 1 << 27


def plasma_species(nphys, device):
    """Species of the plasma + beam workload as (pos, mom, n, q, m, immobile)
    FP32 particle records on `device`: electrons, protons, beam, beam ions."""
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import pack_particles
    out = []
    per_plane = nphys[0] * nphys[1] * 8
    if per_plane * nphys[2] <= STREAM_PARTICLES:
        for sp in I.plasma(nphys, PML, D[0]):
            pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp32", device=device)
            out.append((pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"]))
        return out
    beam, planes = I.plasma_planes(nphys, PML, D[0])
    n = per_plane * nphys[2]
    recs = [(torch.empty((n, 4), dtype=torch.float32, device=device),
             torch.empty((n, 4), dtype=torch.float32, device=device)) for _ in range(2)]
    qm = [None, None]
    for k, el, pr in planes:
        for s_, sp in enumerate((el, pr)):
            pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp32", device="cpu")
            recs[s_][0][k * per_plane:(k + 1) * per_plane].copy_(pos)
            recs[s_][1][k * per_plane:(k + 1) * per_plane].copy_(mom)
            qm[s_] = (sp["q"], sp["m"])
    for s_ in range(2):
        out.append((recs[s_][0], recs[s_][1], n, qm[s_][0], qm[s_][1], False))
    for sp in beam:
        pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp32", device=device)
        out.append((pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"]))
    return out


def run_plasma(args):
    """Throughput on the thermal plasma + drifting beam workload (electrons
    and protons 8 per cell filling the physical box, Maxwellian u_th = 0.01,
    a beam at u_z = 5 with immobile neutralising ions; 16-cell PML, order 1,
    FP32, sort every 20 steps; 128 x 128 x 256 physical cells by default,
    --plasma-cells for smaller profiling captures).  Particles move a small
    fraction of a cell per step and scatter over the whole grid, so the
    particle kernel's current lands on many distinct nodes.  Prints its own
    JSON line; the roofline uses the same byte model as the beam."""
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Sim, pack_particles
    from paper_2201_09084_gb300 import build as B
    B.build()
    nphys = tuple(int(x) for x in args.plasma_cells.split(","))
    species = plasma_species(nphys, "cuda")
    stream = torch.cuda.current_stream()
    sim = Sim(3, nphys, D, PML, cfl=0.99, order=1, prec="fp32", alpha_mode="damped", sort_every=0,
              stream=stream)
    keep = []
    for pos, mom, n, q, m, imm in species:
        sim.add_species(pos, mom, n, q, m, imm)
        keep.append((pos, mom, imm))
    sim.sort()
    if args.tuning:
        p_, k_ = (int(x) for x in args.tuning.split(","))
        sim.set_tuning(p_, k_)
        tuning = {"particles_per_thread": p_, "z_nodes_per_thread": k_, "source": "--tuning"}
    else:
        tuning = sim.autotune(steps=3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    def one_step(i, ev=None):
        if i % SORT_EVERY == 0:
            sim.sort()
        if ev is not None:
            ev[0].record(stream)
        sim.push_deposit()
        if ev is not None:
            ev[1].record(stream)
        sim.field_step()
        if ev is not None:
            ev[2].record(stream)

    for i in range(args.warmup):
        one_step(i)
    sim.sync()
    ps0 = sim.particle_steps()
    l0 = sim.launch_count()
    cells = []
    for pos, mom, imm in keep:
        if not imm:
            c = mom.view(torch.int32)[:, 3]
            cells.append(c[c >= 0])
    occ = int(torch.unique(torch.cat(cells)).numel())
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for i in range(args.steps):
        one_step(args.warmup + i, evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sim.sync()
    ms = t0.elapsed_time(t1)
    psteps = sim.particle_steps() - ps0
    launches = sim.launch_count() - l0
    t_pd = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    t_f = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    N = [n + 2 * p for n, p in zip(nphys, PML[::2])]
    total = N[0] * N[1] * N[2]
    interior = nphys[0] * nphys[1] * nphys[2]
    p_ = tuning["particles_per_thread"]
    b_part, b_field = algorithmic_bytes(psteps / args.steps, occ, interior, total - interior, "fp32", bn=p_ == 2)
    peak, kind = measured_peak()
    achieved = b_part / (t_pd / 1e3) / 1e9
    # measured DRAM bytes per particle of the kernel the launch shape selects
    per_particle = {1: PLASMA_NCU_BYTES_PER_PARTICLE, 2: HEADLINE_NCU_BYTES_PER_PARTICLE}.get(p_)
    traffic = per_particle * psteps / args.steps if per_particle else None
    sim.close()
    return {"metric": METRIC, "value": psteps / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"thermal plasma + drifting beam: {nphys[0]}x{nphys[1]}x{nphys[2]} + "
                                   f"{PML[0]}-cell PML, e- and p+ 8 per cell, u_th 0.01, beam u_z 5, order 1, "
                                   "fp32 fields + float-float PML parts",
                       "particles": int(sum(sp[2] for sp in species if not sp[5])),
                       "sort_every": SORT_EVERY, "l2": "working set > L2"},
            "kernel_ms": {"push_deposit": t_pd, "field_step": t_f},
            "roofline": {"bound": "hbm", "kernel": "push_deposit (particle kernels)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{kind} (copy)",
                         "traffic": traffic, "traffic_note": "per step; ncu of the 64x64x128 case, scaled by particles",
                         "algorithmic_bytes_per_step": b_part,
                         "note": "one launch per mobile species per step; time and bytes are per step"},
            "gpu_launches": int(launches), "autotune": tuning, "clocks": clk}


# ----------------------------------------------------------------------------
# The default workload: the 537M-particle plasma + beam box.
HL_NPHYS = (256, 256, 512)
HL_SMALL = ((24, 24, 48), (8,) * 6)   # the reduced box the oracle steps (cpu_baseline)


def headline_workload(nphys, split64):
    N = [n + 2 * p for n, p in zip(nphys, PML[::2])]
    return {"workload": f"thermal plasma + drifting beam: {nphys[0]}x{nphys[1]}x{nphys[2]} + {PML[0]}-cell PML "
                        f"({N[0]}x{N[1]}x{N[2]} cells), e- and p+ 8 per cell, u_th 0.01, beam u_z 5 into the +z PML, "
                        "order 1, damped PML, sort every 20 steps, fp32 fields and momenta with "
                        + ("IEEE fp64" if split64 else "float-float") + " PML split parts",
            "grid": N, "shape_order": 1, "alpha": "damped (Eq. alpha, v=c)", "sort_every": SORT_EVERY,
            "l2": "working set > L2 (particles 17 GB)", "data": "synthetic (seeded, drawn on the device)"}


def headline_records(nphys, device):
    """Initial records of the default workload as [(pos, mom, n, q, m,
    immobile)] on `device`: electrons and protons drawn on the device, the
    beam and its ions on the host."""
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import pack_particles, pack_records
    out = []
    for sp in I.plasma_device(nphys, PML, D[0], device=device):
        pos, mom = pack_records(sp["cell"], sp["off"], sp["u"], sp["w"])
        out.append((pos, mom, pos.shape[0], sp["q"], sp["m"], False))
        del sp
    torch.cuda.empty_cache()
    for sp in I.plasma_beam(nphys, PML, D[0]):
        pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp32", device=device)
        out.append((pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"]))
    return out


def run_headline(args, rank, world):
    import torch
    from paper_2201_09084_gb300.api import Sim
    from paper_2201_09084_gb300 import build as B

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        torch.distributed.barrier()
    nphys = HL_NPHYS if args.cells is None else tuple(int(x) for x in args.cells.split(","))
    recs = headline_records(nphys, "cuda")
    # the initial records, kept in pinned host memory (reloaded for each run)
    host = []
    for pos, mom, n, q, m, imm in recs:
        hp = torch.empty(pos.shape, dtype=pos.dtype, pin_memory=True)
        hm = torch.empty(mom.shape, dtype=mom.dtype, pin_memory=True)
        hp.copy_(pos)
        hm.copy_(mom)
        host.append((hp, hm))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    n_mobile = sum(r[2] for r in recs if not r[5])
    rec_bytes = sum(2 * r[0].numel() * 4 for r in recs)

    def make(split64, prec="fp32"):
        sim = Sim(3, nphys, D, PML, cfl=0.99, order=1, prec=prec, alpha_mode="damped", sort_every=SORT_EVERY,
                  split_fp64=split64, stream=stream)
        for pos, mom, n, q, m, imm in recs:
            sim.add_species(pos, mom, n, q, m, imm)
        return sim

    def reload():
        for (pos, mom, *_), (hp, hm) in zip(recs, host):
            pos.copy_(hp, non_blocking=True)
            mom.copy_(hm, non_blocking=True)

    def timed(sim, tuning):
        """W untimed steps, then K timed ones (sort every 20 steps inside);
        returns (ms, particle-steps, launches, mean push_deposit ms, mean
        field_step ms, clocks)."""
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

        def one_step(i, ev=None):
            if i % SORT_EVERY == 0:
                sim.sort()
            if ev is not None:
                ev[0].record(stream)
            sim.push_deposit()
            if ev is not None:
                ev[1].record(stream)
            sim.field_step()
            if ev is not None:
                ev[2].record(stream)

        sim.set_tuning(tuning["particles_per_thread"], tuning["z_nodes_per_thread"])
        for i in range(args.warmup):
            one_step(i)
        sim.sync()
        ps0, l0 = sim.particle_steps(), sim.launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = Clocks(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        t0.record(stream)
        for i in range(args.steps):
            one_step(args.warmup + i, evs[i])
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
        sim.sync()
        return (t0.elapsed_time(t1), sim.particle_steps() - ps0, sim.launch_count() - l0,
                float(np.mean([e[0].elapsed_time(e[1]) for e in evs])),
                float(np.mean([e[1].elapsed_time(e[2]) for e in evs])), clk)

    # ---- the measured form: IEEE FP64 PML parts ----
    sim = make(True)
    sim.sort()
    if args.tuning:
        p_, k_ = (int(x) for x in args.tuning.split(","))
        tuning = {"particles_per_thread": p_, "z_nodes_per_thread": k_, "source": "--tuning"}
    else:
        tuning = sim.autotune(steps=3)   # from a restored snapshot
    sim.close()
    reload()
    sim = make(True)
    ms, psteps, launches, t_pd, t_f, clk = timed(sim, tuning)
    sim.close()

    # ---- end to end: the records uploaded from pinned host memory inside the timed region ----
    sim = make(True)
    sim.set_tuning(tuning["particles_per_thread"], tuning["z_nodes_per_thread"])
    torch.cuda.synchronize()
    nsteps_e2e = args.warmup + args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reload()
    for _ in range(nsteps_e2e):
        sim.step(1)
        ps_e2e = sim.particle_steps()   # each step's result read back (synchronising 8-byte copy)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    sim.close()

    # ---- the same run with float-float PML parts ----
    ff = None
    if not args.no_extra:
        reload()
        sim = make(False)
        ms2, ps2, _, t_pd2, t_f2, _ = timed(sim, tuning)
        sim.close()
        ff = {"value": ps2 / (ms2 / 1e3), "unit": "particle-steps/s", "ms_per_step": ms2 / args.steps,
              "kernel_ms": {"push_deposit": t_pd2, "field_step": t_f2}}
        # the deterministic form: int64 fixed-point deposition (same launch shapes)
        reload()
        sim = make(True, prec="fixed64")
        ms3, ps3, _, t_pd3, t_f3, _ = timed(sim, tuning)
        sim.close()
        fx = {"value": ps3 / (ms3 / 1e3), "unit": "particle-steps/s", "ms_per_step": ms3 / args.steps,
              "kernel_ms": {"push_deposit": t_pd3, "field_step": t_f3},
              "note": "int64 fixed-point deposition (bit-identical under any particle order), IEEE fp64 PML parts"}
    del recs, host
    torch.cuda.empty_cache()

    ms, psteps, ms_e2e, ps_e2e = combine_ranks(ms, psteps, ms_e2e, ps_e2e, world, "cuda")
    N = [n + 2 * p for n, p in zip(nphys, PML[::2])]
    total = N[0] * N[1] * N[2]
    interior = nphys[0] * nphys[1] * nphys[2]
    n_live = (psteps / world) / args.steps
    # occupied cells: the plasma fills every physical cell
    p_ = tuning["particles_per_thread"]
    b_part, b_field = algorithmic_bytes(n_live, interior, interior, total - interior, "fp32", bn=p_ == 2)
    peak, kind = measured_peak()
    achieved = b_part / (t_pd / 1e3) / 1e9
    traffic = (HEADLINE_NCU_BYTES_PER_PARTICLE * n_live
               if HEADLINE_NCU_BYTES_PER_PARTICLE and p_ == 2 else None)
    kname = ("k_tile (tile-resident fused gather/push/move/deposit/damp)" if p_ == 2
             else "particle kernels (fused gather/push/move/deposit/damp)")
    out = {
        "metric": METRIC, "value": psteps / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(headline_workload(nphys, True), particles=int(n_mobile), parallelism=f"replicas x{world}"),
        "cell_updates_per_s": world * total * args.steps / (ms / 1e3),
        "kernel_ms": {"push_deposit": t_pd, "field_step": t_f},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{kind} (copy)", "traffic": traffic,
                     "traffic_note": HEADLINE_NCU_NOTE if traffic else None,
                     "algorithmic_bytes_per_launch": b_part,
                     "bytes_model": ("60 B per live particle (32 read, 28 written) + 36 B per occupied cell "
                                     "(E and B at the integer time read, J written)") if p_ == 2 else
                                    ("60 B per live particle (32 read, 28 written) + 48 B per occupied cell "
                                     "(9 field words read, 3 current words written)")},
        "e2e": {"value": ps_e2e / (ms_e2e / 1e3), "unit": "particle-steps/s",
                "h2d_bytes_per_step": rec_bytes / nsteps_e2e, "d2h_bytes_per_step": 8,
                "note": f"the initial particle records ({rec_bytes / 1e9:.1f} GB) copied from pinned host memory "
                        f"once per run of {nsteps_e2e} steps (h2d bytes are that copy per step); every step runs "
                        "step_n (sorting every 20 steps) and reads its particle-step count back to the host"},
        "gpu_launches": int(launches),
        "autotune": tuning,
        "clocks": clk,
    }
    if ff is not None:
        out["float_float_parts"] = ff
        out["deterministic_fixed64"] = fx
        out["fixed64_over_fp32"] = fx["value"] / out["value"]
    return out


def cpu_plasma_sample(steps, gpu_check=True, threads=None):
    """The oracle on the plasma + beam workload reduced to 24 x 24 x 48
    physical cells + 8-cell PML (221,186 mobile particles; the same
    distributions, beam radius 4 and length 12 cells), `steps` steps on the
    host's cores.  Returns (particle-steps/s, threads used, description,
    ms per step, max relative field error of the GPU's FP32 form on the same
    sample or None)."""
    import oracle as O
    from paper_2201_09084_gb300 import inputs as I
    O.build()
    nphys, pml = HL_SMALL
    parts = I.plasma(nphys, pml, D[0], beam_radius=4.0, beam_length=12.0)
    dt = O.yee_dt(D, 0.99, 3)
    nthreads = O.set_threads(threads)
    ora = O.OracleSim(3, nphys, pml, D, dt, order=1, alpha_mode="damped")
    for sp in parts:
        X = I.absolute(sp["cell"], sp["off"])
        u = sp["u"].astype(np.float64)
        ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], sp["w"].astype(np.float64),
                          sp["q"], sp["m"], sp["immobile"])
    nmob = int(sum(len(sp["w"]) for sp in parts if not sp["immobile"]))
    t = 0.0
    psteps = 0
    for _ in range(steps):
        psteps += int(np.count_nonzero(ora.particles()["alive"][:nmob]))
        a = time.perf_counter()
        ora.step(1)
        t += time.perf_counter() - a
    desc = (f"FP64 C oracle, {nthreads} threads: the workload reduced to {nphys[0]}x{nphys[1]}x{nphys[2]} + "
            f"{pml[0]}-cell PML ({nmob} mobile particles), {steps} steps")
    err = None
    if gpu_check:
        import torch
        from paper_2201_09084_gb300.api import Sim, pack_particles
        gpu = Sim(3, nphys, D, pml, dt=dt, order=1, prec="fp32", alpha_mode="damped", sort_every=SORT_EVERY,
                  split_fp64=True)
        keep = []
        for sp in parts:
            pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp32")
            gpu.add_species(pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"])
            keep.append((pos, mom))
        gpu.set_tuning(2, 1)
        gpu.step(steps)
        gpu.sync()
        names = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
        unit = {k: (O.C_LIGHT if k[0] == "B" else 1.0) for k in names}
        a_ = {k: ora.field(k) * unit[k] for k in names}
        b_ = {k: gpu.field(k).cpu().numpy() * unit[k] for k in names}
        scale = max(np.abs(v).max() for v in a_.values())
        err = float(max(np.abs(a_[k] - b_[k]).max() for k in names) / scale)
        gpu.close()
    return psteps / t, nthreads, desc, 1e3 * t / steps, err


# ----------------------------------------------------------------------------
# The cavity run of Sec. III: a pillbox cavity on a beam pipe (zeroed-field
# cells), 10-cell PMLs on the z faces only with delta = 10 cells, a proton
# beam injected continuously inside the undamped entry face's PML.
CAV_NPHYS = (64, 64, 108)
CAV_PML = (0, 0, 0, 0, 10, 10)
CAV_D = (1e-3, 1e-3, 1e-3)


def run_cavity(args):
    """Throughput of the cavity workload (own JSON line): 64 x 64 x 108
    cells of 1 mm + 10-cell z PMLs (sigma with delta = 10 cells), Yee at
    0.99 x c dt = d / sqrt(3), conducting x and y walls; a pillbox cavity
    (radius 30 cells, 40 cells long) on a beam pipe (radius 10 cells) carved
    out by zeroed-field cells; a 40 nC, gamma = 479 proton beam injected
    continuously (1,000 macroparticles per step over the first `steps`
    steps) inside the -z PML, which deposits undamped, and leaving through
    the damped +z PML; order 1, FP32 with float-float PML parts.  Every step
    is an injection (pic_inject) plus step_n(1)."""
    import torch
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Sim, pack_particles
    from paper_2201_09084_gb300 import build as B
    B.build()
    stream = torch.cuda.current_stream()
    faces = ["damped", "damped", "damped", "damped", "one", "damped"]
    per = 1000
    nsl = args.warmup + args.steps

    def make():
        sim = Sim(3, CAV_NPHYS, CAV_D, CAV_PML, cfl=0.99, order=1, prec="fp32", alpha_mode="damped", delta=10.0,
                  face_alpha=faces, stream=stream)
        sim.set_conductor(I.cavity_mask(CAV_NPHYS, CAV_PML, pipe_radius=10, cavity_radius=30, cavity_z=(34, 74)))
        cap = nsl * per
        z = np.zeros((cap, 3))
        pos0, mom0 = pack_particles(z.astype(np.int64), z.astype(np.float32), z.astype(np.float32),
                                    np.zeros(cap, np.float32), "fp32")
        sid = sim.add_species(pos0, mom0, 0, I.Q_E, I.M_P)
        return sim, sid

    sim, sid = make()
    shift = 299792458.0 * sim.dt / CAV_D[2] * np.sqrt(1 - 1 / 479.0 ** 2)
    b = I.cavity_beam_slices(CAV_NPHYS, CAV_PML, nsl, per, shift, sigma=3.0)
    pos, mom = pack_particles(b["cell"], b["off"], b["u"], b["w"], "fp32")
    for st in range(args.warmup):
        sim.inject(sid, pos[st * per:(st + 1) * per], mom[st * per:(st + 1) * per])
        sim.step(1)
    sim.sync()
    ps0, l0 = sim.particle_steps(), sim.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for st in range(args.warmup, nsl):
        sim.inject(sid, pos[st * per:(st + 1) * per], mom[st * per:(st + 1) * per])
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sim.sync()
    ms = e0.elapsed_time(e1)
    psteps = sim.particle_steps() - ps0
    launches = sim.launch_count() - l0
    N = [n + CAV_PML[2 * a] + CAV_PML[2 * a + 1] for a, n in enumerate(CAV_NPHYS)]
    total = N[0] * N[1] * N[2]
    interior = CAV_NPHYS[0] * CAV_NPHYS[1] * CAV_NPHYS[2]
    _, b_field = algorithmic_bytes(0, 0, interior, total - interior, "fp32")
    peak, kind = measured_peak()
    achieved = (b_field + 60 * psteps / args.steps) / (ms / args.steps / 1e3) / 1e9
    sim.close()
    return {"metric": METRIC, "value": psteps / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cavity run (Sec. III): 64x64x108 cells of 1 mm + 10-cell z PMLs (delta 10 "
                                   "cells), pillbox cavity r=30 on a beam pipe r=10 (zeroed-field cells), 40 nC "
                                   "gamma 479 proton beam injected continuously in the undamped -z PML, damped +z "
                                   "PML, order 1, fp32 + float-float PML parts",
                       "cells": total, "injected_per_step": per},
            "cell_updates_per_s": total * args.steps / (ms / 1e3),
            "roofline": {"bound": "hbm", "kernel": "whole step (inject, particles, E pass, conductor, B pass)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": f"{kind} (copy)", "traffic": None,
                         "note": "field bytes per step (60 B per interior cell, 228 B per PML cell) plus 60 B per "
                                 "pushed particle, over the step time; the 0.56 M-cell box fits in L2, so the "
                                 "step is launch- and latency-bound"},
            "gpu_launches": int(launches), "clocks": clk}


def run_reference_plasma(args, rank, world):
    """The reference arm: the FP64 oracle on the default workload reduced to
    the sample cpu_plasma_sample() steps (bounded: W + K steps), timed on the
    host's cores; rank 0 only."""
    if rank != 0:
        return None
    v, nthreads, desc, ms_step, _ = cpu_plasma_sample(args.warmup + args.steps, gpu_check=False)
    cfg = dict(headline_workload(HL_NPHYS, True), parallelism="cpu oracle",
               sample=desc + "; the GPU line runs the full 256x256x512 box")
    return {"metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": nthreads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cells", default=None,
                    help="physical cells of the default plasma workload (default 256,256,512; smaller only for "
                         "profiling captures)")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only (no float-float form, beam, batched runs)")
    ap.add_argument("--beam", action="store_true",
                    help="the 3D beam workload (128^3 + 16, 4,194,304 particles) as the main line")
    ap.add_argument("--order", type=int, default=1, choices=[1, 3])
    ap.add_argument("--theta", type=float, default=0.0)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 2D runs measurement")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 run of the beam workload")
    ap.add_argument("--batch-runs", type=int, default=4096, help="number of batched 2D runs")
    ap.add_argument("--particles", type=int, default=NPART,
                    help="beam macroparticles (default 4194304; smaller only for profiling captures)")
    ap.add_argument("--precision-study", action="store_true",
                    help="FP32 forms vs FP64 on the plasma + beam workload (prints its own JSON line)")
    ap.add_argument("--plasma", action="store_true",
                    help="throughput on the host-drawn plasma + beam workload (prints its own JSON line)")
    ap.add_argument("--plasma-cells", default="128,128,256", help="physical cells of the --plasma workload")
    ap.add_argument("--single-particle", action="store_true",
                    help="the 2D FP64 single-particle workload (run it with --steps 400; own JSON line)")
    ap.add_argument("--cavity", action="store_true",
                    help="the cavity workload of Sec. III (zeroed-field cells, injected beam; own JSON line)")
    ap.add_argument("--tuning", default=None,
                    help="P,KZ launch shapes instead of the autotuner (profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.precision_study:
        out = run_precision_study(args) if rank == 0 else None
    elif args.plasma and args.impl == "gb300":
        out = run_plasma(args) if rank == 0 else None
    elif args.single_particle and args.impl == "gb300":
        out = run_single_particle(args) if rank == 0 else None
    elif args.cavity and args.impl == "gb300":
        out = run_cavity(args) if rank == 0 else None
    elif args.impl == "reference":
        out = run_reference(args, rank, world) if args.beam else run_reference_plasma(args, rank, world)
    elif args.beam:
        out = run_beam_line(args, rank, world)
    else:
        out = run_headline(args, rank, world)
        if not args.no_extra:
            b = argparse.Namespace(**vars(args))
            b.tuning, b.no_batch, b.no_cpu_baseline = None, True, True
            ob = run_beam_line(b, rank, world)
            out["beam_3d"] = {"workload": ob["config"]["workload"], "value": ob["value"], "unit": ob["unit"],
                              "ms_per_step": ob["ms_per_step"], "kernel_ms": ob["kernel_ms"],
                              "roofline_frac": ob["roofline"]["frac"], "autotune": ob["autotune"],
                              "fp64": ob.get("fp64"), "fp32_over_fp64": ob.get("fp32_over_fp64")}
            if not args.no_batch:
                out["batch2d"] = batch_lines(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            v, nthreads, desc, _, err = cpu_plasma_sample(SORT_EVERY)
            v1 = cpu_plasma_sample(SORT_EVERY, gpu_check=False, threads=1)[0]
            out["cpu_baseline"] = {"value": v, "unit": "particle-steps/s", "cores": nthreads, "kind": "oracle",
                                   "sample": desc, "value_1_thread": v1,
                                   "gpu_max_rel_field_error_on_sample": err,
                                   "gpu_error_note": "the GPU's FP32 form (tile kernel, IEEE fp64 PML parts) on "
                                                     "the same sample and steps: max |GPU - oracle| over the six "
                                                     "components / max(|E|, c|B|)"}
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def batch_lines(args, rank, world):
    """Batched 2D runs in FP32 and FP64 (each under its CUDA graph), with the
    oracle on a sample of them (rank 0, N=1)."""
    nb = min(args.steps, 200)
    out = {"fp32": run_batch(nb, 3, "fp32", nruns=args.batch_runs),
           "fp64": run_batch(nb, 3, "fp64", nruns=args.batch_runs)}
    out["fp32_over_fp64_particle_steps"] = (out["fp32"]["particle_steps_per_s"] /
                                            out["fp64"]["particle_steps_per_s"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        bv, bc, bdesc = cpu_batch_sample(nruns=args.batch_runs)
        out["cpu_baseline"] = {"value": bv, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                               "sample": bdesc, "cell_updates_per_s": bc}
    return out


def run_beam_line(args, rank, world):
    """The 3D beam workload (128^3 + 16-cell PML, 4,194,304 particles) in FP32
    with the FP64 form beside it."""
    out = run_gpu(args, rank, world)
    if args.prec == "fp32" and not args.no_fp64:
        a64 = argparse.Namespace(**vars(args))
        a64.prec, a64.tuning = "fp64", None
        o64 = run_gpu(a64, rank, world)
        out["fp64"] = {"value": o64["value"], "unit": o64["unit"], "ms_per_step": o64["ms_per_step"],
                       "kernel_ms": o64["kernel_ms"], "autotune": o64["autotune"],
                       "roofline_frac": o64["roofline"]["frac"], "e2e": o64["e2e"]["value"]}
        out["fp32_over_fp64"] = out["value"] / o64["value"]
    if not args.no_batch:
        out["batch2d"] = batch_lines(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, _ = cpu_sample(args.order, args.theta, 65536, 8)
        out["cpu_baseline"] = {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                               "sample": desc}
    return out


if __name__ == "__main__":
    main()
