#!/usr/bin/env python3
"""Throughput of the PIC step on a GB300: cell-updates/s and particle-pushes/s.

Workload (default): 2D, 4096 x 1024 cells, k0 dx1 = 2 pi/32, dx2 = 4 dx1,
dt = dx1/2; Gaussian laser (w0 = 20/k0, sin^2 envelope of 10 wavelengths,
a0 = 4) entering a uniform plasma n = 0.01 n_c that fills x1 in [255, 3840)
cells with 8 electrons per cell (29,368,320 electrons, seeded uniform
positions, thermal momenta u_th = 0.001), immobile ions, quadratic shapes,
customised 16-coefficient solver, Boris pusher.  The headline runs FP32 fields
with the FP64 pusher ("mixed"); the plain FP64 path is measured in the same
run and reported beside it.

One JSON line on stdout (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_03754_gb300 import inputs  # noqa: E402

METRIC = "particle-pushes/s"
FP64_FLOP_PER_PUSH = 70   # 2D Boris (58) + gamma (7) + position update (5), FMA = 2 FLOP
# field update per cell, M = 16 (FMA = 2 FLOP): four 16-tap symmetric-difference x1 stencils
# (16 subtractions + 16 FMA = 48 FLOP each) plus the Yee differences, current term and updates
FIELD_FLOP_PER_CELL = {2: 214, 3: 226}
FP64_PEAK_TFLOPS_AT_MAX = 304 * 2 * 2070e6 / 1e12   # 304 DFMA/cycle/GPU at 2070 MHz
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch from ncu, per
# push: the particle kernel on the 2048x512 workload (python bench.py --small, launch 4),
# scaled to the bench workload's launch (traffic grows with the particles)
PARTICLE_KERNEL_TRAFFIC_PER_PUSH = (366.734592e6 + 240.926464e6) / 6295552
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch: particle "
                  "kernel on the 2048x512 case (6,295,552 electrons) scaled by the particles to "
                  "this launch")
WORKLOAD = "2D 4096x1024 plasma 8ppc a0=4, customised M=16 solver, Boris"


SMALL = False   # --small: 2048 x 512 cells, plasma in [255, 1792) (for profiler captures)


def workload_arrays(seed=inputs.DEFAULT_SEED, ppc=8, frac=1.0):
    n = (2048, 512) if SMALL else (4096, 1024)
    dx = (inputs.DX1, inputs.DX2)
    P = inputs.plasma(n, dx, ppc, (255, n[0] - 256), density=0.01, uth=0.001, seed=seed)
    if frac < 1.0:
        g = inputs.rng(seed + 1)
        keep = np.sort(g.choice(P.n, size=max(1, int(P.n * frac)), replace=False))
        P = inputs.ParticleSet([v[keep] for v in P.x], [v[keep] for v in P.u], P.w[keep])
    return n, dx, P


def c3_workload_arrays(seed=inputs.DEFAULT_SEED, small=False):
    """3D 1024 x 256 x 256, dx2 = dx3 = 4 dx1, cold plasma n = 0.005 n_c, 2 electrons per
    cell in x1 in [255, 896) cells (84,017,152 electrons).  small: 512 x 128 x 128 with
    the plasma in [255, 448) (profiling size)."""
    n = (512, 128, 128) if small else (1024, 256, 256)
    dx = (inputs.DX1, inputs.DX2, inputs.DX2)
    P = inputs.plasma(n, dx, 2, (255, 448) if small else (255, 896), density=0.005, uth=0.0,
                      seed=seed)
    return n, dx, P


def c3_laser_kwargs(n, dx):
    return dict(a0=10.0, k0=1.0, phase=0.0, L_env=20 * np.pi, x_front=255 * dx[0], w0=30.0,
                x2c=n[1] * dx[1] / 2, x3c=n[2] * dx[2] / 2)


def laser_kwargs(n, dx):
    return dict(a0=4.0, k0=1.0, phase=0.0, L_env=20 * np.pi, x_front=255 * dx[0], w0=20.0,
                x2c=n[1] * dx[1] / 2)


def coeff_table():
    from paper_2004_03754_gb300 import coeffs
    return coeffs.load("proposed", 16, 0.5, 0.3)


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self, dev=0):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        rows = [[c.strip() for c in r] for r in rows if r and r[0].strip() == str(dev)]
        if not rows:
            return out
        mhz = [float(r[1].split()[0]) for r in rows if r[1].split()[0].replace(".", "").isdigit()]
        if mhz:
            out["sm_mhz"] = float(np.median(mhz))
        try:
            out["sm_max_mhz"] = float(rows[0][2].split()[0])
        except Exception:
            pass
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for i, nm in enumerate(names):
            if any(len(r) > 5 + i and r[5 + i].lower().startswith("active") for r in rows):
                out["reasons"].append(nm)
        return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def max_over_ranks(ms_local, dist=None, device="cuda"):
    """Duration of the timed region on the slowest rank (ms), returned on every
    rank (all-reduce MAX; the identity on one process)."""
    if dist is None:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, ms_max):
    """Units all ranks processed per second of the slowest rank's timed region:
    every rank advances the same workload (replicas, weak scaling)."""
    return units_per_rank_step * steps * world / (ms_max / 1e3)


def run_gpu(args):
    import torch
    from paper_2004_03754_gb300 import pic as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n, dx, Pset = workload_arrays()
    cE, cB = coeff_table()
    dt = inputs.DT
    stream = torch.cuda.Stream()
    res = {}

    def one(precision, steps, warmup, clocks_path=None):
        sim = P.Simulation(n, dx, dt, cE, cB, precision=precision, pusher="boris",
                           stream=stream.cuda_stream)
        sim.load_laser(**laser_kwargs(n, dx))
        sim.load_particles(Pset.x, Pset.u, Pset.w, Pset.qm)
        sim.step(warmup)
        sim.sync()
        info = sim.info()
        if dist:
            dist.barrier()
        P.pic_set_timing(sim.ctx, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx = Clocks(clocks_path) if clocks_path else None
        if ctx:
            ctx.__enter__()
            time.sleep(0.3)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if ctx:
            ctx.__exit__()
        ms = e0.elapsed_time(e1)
        t = P.pic_get_timing(sim.ctx)
        P.pic_set_timing(sim.ctx, False)
        sim.sync()
        clocks = ctx.summary(local) if ctx else None
        out = dict(ms=ms, timing=t, info=info, clocks=clocks, sim=sim)
        return out

    steps, warmup = args.steps, args.warmup
    clocks_csv = args.clocks_csv or os.path.join(tempfile.gettempdir(),
                                                 "pic_bench_clocks_rank%d.csv" % local)
    mixed = one("mixed", steps, warmup, clocks_csv)
    ms_local = max_over_ranks(mixed["ms"], dist, "cuda")
    ms_step = ms_local / steps
    npart = Pset.n
    ncell = n[0] * n[1]
    value = whole_job_rate(npart, steps, world, ms_local)
    cells_s = whole_job_rate(ncell, steps, world, ms_local)
    t = mixed["timing"]
    # roofline of the dominant kernel (particles).  Its binding resource is the
    # FP64 pipe (GB300: 2 DFMA/clk/SM): algorithmic FP64 work per push is the
    # Boris rotation, gamma and the position update, 70 FLOP (FMA = 2).  The
    # HBM view (88 algorithmic bytes per push) is reported beside it.
    part_ms = t.ms_particles / steps
    alg_bytes = 88.0 * npart
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (part_ms / 1e3) / 1e9
    sm_mhz = (mixed["clocks"] or {}).get("sm_mhz") or 2070.0
    fp64_peak = 304 * 2 * sm_mhz * 1e6 / 1e12          # TFLOP/s at the sampled clock
    fp64_ach = FP64_FLOP_PER_PUSH * npart / (part_ms / 1e3) / 1e12
    fld_ms = t.ms_fields / steps
    fld_gbs = 60.0 * ncell / (fld_ms / 1e3) / 1e9
    sim = mixed["sim"]

    # end to end through the public API with pinned host buffers: per step the
    # particle state is loaded from the host, advanced one step and read back
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(np.concatenate(Pset.x)).pin_memory()
        Uh = torch.from_numpy(np.concatenate(Pset.u)).pin_memory()
        Wh = torch.from_numpy(Pset.w.copy()).pin_memory()
        Xo = torch.empty_like(Xh).pin_memory()
        Uo = torch.empty_like(Uh).pin_memory()
        e2e_steps = max(2, min(steps, 5))
        P.pic_load_particles(sim.ctx, npart, Xh, Uh, Wh, -1.0)
        P.pic_step(sim.ctx, 1)
        P.pic_read_particles(sim.ctx, Xo, Uo, None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            P.pic_load_particles(sim.ctx, npart, Xh, Uh, Wh, -1.0)
            P.pic_step(sim.ctx, 1)
            P.pic_read_particles(sim.ctx, Xo, Uo, None)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": npart * e2e_steps / el, "unit": METRIC,
               "h2d_bytes_per_step": int(Xh.numel() * 8 + Uh.numel() * 8 + Wh.numel() * 8),
               "d2h_bytes_per_step": int(Xo.numel() * 8 + Uo.numel() * 8)}
    sim.close()
    mixed["sim"] = None

    fp64 = None
    if not args.no_fp64:
        r = one("fp64", max(3, steps // 2), warmup)
        t64 = r["timing"]
        s64 = max(3, steps // 2)
        f64_fld = FIELD_FLOP_PER_CELL[2] * ncell / (t64.ms_fields / s64 / 1e3) / 1e12
        f64_par = FP64_FLOP_PER_PUSH * npart / (t64.ms_particles / s64 / 1e3) / 1e12
        fp64 = {"particle_pushes_per_s": npart * s64 / (r["ms"] / 1e3),
                "cell_updates_per_s": ncell * s64 / (r["ms"] / 1e3),
                "ms_per_step": r["ms"] / s64,
                "particle_kernel_ms": t64.ms_particles / s64,
                "field_kernel_ms": t64.ms_fields / s64,
                # both kernels are bound by the FP64 pipe in this form
                "field_kernel_roofline": {"bound": "alu", "achieved": f64_fld, "peak": fp64_peak,
                                          "unit": "TFLOP/s (FP64)", "frac": f64_fld / fp64_peak,
                                          "alg_flop_per_cell": FIELD_FLOP_PER_CELL[2]},
                # push, gamma and move only: in this form the gather and the deposit run in
                # FP64 as well and are not counted, so this is a lower bound on the FP64 use
                "particle_kernel_push_flop_view": {"achieved": f64_par, "peak": fp64_peak,
                                                   "unit": "TFLOP/s (FP64)", "frac": f64_par / fp64_peak,
                                                   "alg_flop_per_push": FP64_FLOP_PER_PUSH}}
        r["sim"].close()

    comp = None
    if not args.no_fp64:
        s_c = max(3, steps // 2)
        r = one("compensated", s_c, warmup)
        tc = r["timing"]
        comp = {"particle_pushes_per_s": npart * s_c / (r["ms"] / 1e3),
                "cell_updates_per_s": ncell * s_c / (r["ms"] / 1e3),
                "ms_per_step": r["ms"] / s_c,
                "particle_kernel_ms": tc.ms_particles / s_c,
                "field_kernel_ms": tc.ms_fields / s_c,
                "field_kernel_gbs_alg": 120.0 * ncell / (tc.ms_fields / s_c / 1e3) / 1e9,
                "precision": "f32-pair (48-bit) fields, f64 pusher, f32 current"}
        if fp64:
            comp["speedup_vs_fp64"] = fp64["ms_per_step"] / comp["ms_per_step"]
        r["sim"].close()

    ensemble = None
    if not args.no_ensemble:
        ensemble = run_ensemble(stream)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(stream)
    c1 = None
    if not args.no_c1:
        c1 = run_c1(stream)
    c3 = None
    if not args.no_c3:
        c3 = c3_leg(stream, fp64=not args.no_fp64)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 fields + f64 pusher", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": list(n), "particles": npart,
                   "ppc": 8, "precision": "mixed", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (particle state 1.4 GB)"},
        "cell_updates_per_s": cells_s,
        "kernel_ms_per_step": {"rebin": t.ms_rebin / steps, "particles": part_ms,
                               "stragglers": t.ms_stragglers / steps,
                               "correction": t.ms_correction / steps, "fields": fld_ms},
        "roofline": {"bound": "alu", "kernel": "particle_kernel<float,2>",
                     "achieved": fp64_ach, "peak": fp64_peak, "unit": "TFLOP/s (FP64)",
                     "frac": fp64_ach / fp64_peak,
                     "traffic": PARTICLE_KERNEL_TRAFFIC_PER_PUSH * npart,
                     "traffic_source": TRAFFIC_SOURCE,
                     "alg_flop_per_launch": FP64_FLOP_PER_PUSH * npart,
                     "peak_derivation": "304 DFMA/cycle/GPU x 2 FLOP x sampled SM clock",
                     "hbm_view": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "peak_kind": peak_kind,
                                  "alg_bytes_per_launch": alg_bytes}},
        "field_kernel_roofline": {"bound": "hbm", "kernel": "field_march_kernel<float,16>",
                                  "achieved": fld_gbs, "peak": peak, "unit": "GB/s",
                                  "frac": fld_gbs / peak, "alg_bytes_per_cell": 60,
                                  "traffic": None,
                                  "traffic_source": "not captured for the current field kernel "
                                                    "(J read into registers since the last capture)"},
        "fp64_plain": fp64,
        "compensated": comp,
        "ensemble": ensemble,
        "adjoint": adjoint,
        "c1": c1,
        "c3": c3,
        "e2e": e2e,
        "gpu_launches": int(t.launches),
        "sort_interval": mixed["info"].sort_interval,
        "clocks": mixed["clocks"],
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# Ensemble: 256 independent 2D vacuum runs in one persistent launch
# --------------------------------------------------------------------------
N_CAP = 8192


def ensemble_setup(nruns=256, seed=inputs.DEFAULT_SEED):
    """Grids n1 ~ U{256..2048}, n2 ~ U{64..256}; a0 log-uniform in [10, 1e4]; plane-wave
    sin^2 pulse of min(10 wavelengths, n1/2 cells); 16 electrons at rest at
    front + 16 + 2i cells, x2 = (i+1/2) n2/16; steps = the pulse's passage over the
    last electron, int(L(1 + 3 a0^2/32) + distance)/dt, capped at N_CAP."""
    n1, n2, a0 = inputs.ensemble(nruns, seed)
    dx1, dx2, dt = inputs.DX1, inputs.DX2, inputs.DT
    lasers, counts, xs1, xs2, steps = [], [], [], [], []
    for r in range(nruns):
        Lc = min(320, int(n1[r]) // 2)
        Lenv = Lc * dx1
        xf = (Lc + 4) * dx1
        lasers.append(dict(a0=float(a0[r]), k0=1.0, phase=0.0, L_env=Lenv, x_front=xf, w0=0.0,
                           x2c=n2[r] * dx2 / 2))
        for i in range(16):
            xs1.append(xf + (16 + 2 * i) * dx1)
            xs2.append((i + 0.5) * n2[r] * dx2 / 16)
        counts.append(16)
        t_pass = Lenv * (1 + 3 * a0[r] ** 2 / 32) + 50 * dx1
        steps.append(int(min(math.ceil(t_pass / dt), N_CAP)))
    return n1, n2, a0, lasers, counts, [np.array(xs1), np.array(xs2)], np.array(steps)


def _ensemble_once(stream, precision, n1, n2, a0, lasers, counts, x, steps):
    from paper_2004_03754_gb300 import pic as P
    cE, cB = coeff_table()
    npart = int(sum(counts))
    ens = P.Ensemble(n1, n2, (inputs.DX1, inputs.DX2), inputs.DT, cE, cB, precision=precision,
                     pusher="analytic", stream=stream.cuda_stream)
    ens.autotune(8)
    ens.load_lasers([P.pic_laser(l["a0"], l["k0"], l["phase"], l["L_env"], l["x_front"], l["w0"],
                                 l["x2c"], 0.0) for l in lasers])
    ens.load_particles(counts, x, [np.zeros(npart)] * 3, np.zeros(npart))
    ens.set_steps(steps)
    ens.run()
    info = ens.info()
    _, ug, _ = ens.read_particles()
    ens.close()
    sec = info.last_run_ms / 1e3
    bytes_per_cell = 48.0 if precision == "mixed" else 96.0   # E, B read and written
    return {"ms": info.last_run_ms, "tile": list(info.tile), "graph": bool(info.graph),
            "grid_blocks": info.grid_blocks,
            "cell_updates_per_s": info.cell_steps / sec,
            "particle_pushes_per_s": info.particle_steps / sec,
            "field_hbm_gbs": bytes_per_cell * info.cell_steps / sec / 1e9,
            "cell_steps": int(info.cell_steps), "steps_max": int(info.max_steps),
            "total_cells": int(info.total_cells)}, np.sqrt(1 + ug[0] ** 2 + ug[1] ** 2 + ug[2] ** 2)


def run_ensemble(stream, seq_sample=4, fp64_check=6):
    """C4: the 256-run ensemble in one persistent launch per precision -- FP32
    fields ("mixed"), compensated FP32-pair fields and FP64 -- each against the
    same runs on the plain FP64 path one after another, and each electron's
    energy against the plain FP64 path over the a0 range."""
    from paper_2004_03754_gb300 import pic as P
    n1, n2, a0, lasers, counts, x, steps = ensemble_setup()
    cE, cB = coeff_table()
    forms = {"mixed": "f32 fields + f64 analytic pusher",
             "compensated": "f32-pair (48-bit) fields + f64 analytic pusher",
             "fp64": "f64 fields + f64 analytic pusher"}
    out = {"runs": len(n1), "capped_fraction": float(np.mean(steps >= N_CAP)), "forms": {}}
    gam = {}
    for prec, desc in forms.items():
        # the FP64 ensemble is timed on the first 1024 steps of every run (its
        # accuracy is the oracle's, checked by the tests); the reduced forms run
        # the whole workload so that their energies can be compared below
        st = np.minimum(steps, 1024) if prec == "fp64" else steps
        r, gam[prec] = _ensemble_once(stream, prec, n1, n2, a0, lasers, counts, x, st)
        r["precision"] = desc
        if prec == "fp64":
            r["steps_timed"] = "min(steps, 1024) per run"
        out["forms"][prec] = r
    out["total_cells"] = out["forms"]["mixed"]["total_cells"]
    out["steps_max"] = out["forms"]["mixed"]["steps_max"]
    # the same runs on the plain FP64 path, one context per run, sequentially:
    # a sample of runs, extrapolated by cell-steps
    rng = inputs.rng(5)
    pick = rng.choice(len(n1), seq_sample, replace=False)
    t_seq, cs_seq = 0.0, 0
    import torch
    for r in pick:
        sim = P.Simulation((int(n1[r]), int(n2[r])), (inputs.DX1, inputs.DX2), inputs.DT, cE, cB,
                           precision="fp64", pusher="analytic", stream=stream.cuda_stream)
        sim.load_laser(**lasers[r])
        o = int(sum(counts[:r]))
        sim.load_particles([x[0][o:o + 16], x[1][o:o + 16]], [np.zeros(16)] * 3, np.zeros(16))
        ns = min(int(steps[r]), 512)
        sim.step(2)
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(ns)
        e1.record(stream)
        torch.cuda.synchronize()
        t_seq += e0.elapsed_time(e1) / 1e3
        cs_seq += int(n1[r]) * int(n2[r]) * ns
        sim.close()
    seq_rate = cs_seq / t_seq
    out["fp64_sequential_cell_updates_per_s"] = seq_rate
    for prec in forms:
        out["forms"][prec]["speedup_vs_fp64_sequential"] = out["forms"][prec]["cell_updates_per_s"] / seq_rate
    # single-electron energy of each form against the plain FP64 path (itself
    # checked against the oracle at 1e-12) over the a0 range: relative error of the
    # mean kinetic energy gamma - 1 of the run's 16 electrons after its last step
    order = np.argsort(a0)
    sel = order[np.linspace(0, len(order) - 1, fp64_check).astype(int)]
    errs = []
    for r in sel:
        sim = P.Simulation((int(n1[r]), int(n2[r])), (inputs.DX1, inputs.DX2), inputs.DT, cE, cB,
                           precision="fp64", pusher="analytic", stream=stream.cuda_stream)
        sim.load_laser(**lasers[r])
        o = int(sum(counts[:r]))
        sim.load_particles([x[0][o:o + 16], x[1][o:o + 16]], [np.zeros(16)] * 3, np.zeros(16))
        sim.step(int(steps[r]))
        _, uu, _ = sim.read_particles()
        sim.close()
        g64 = np.sqrt(1 + uu[0] ** 2 + uu[1] ** 2 + uu[2] ** 2)
        e64 = float(np.mean(g64 - 1))
        row = {"a0": float(a0[r]), "steps": int(steps[r]), "energy_fp64": e64}
        for prec in ("mixed", "compensated"):
            eb = float(np.mean(gam[prec][o:o + 16] - 1))
            row["rel_err_" + prec] = abs(eb - e64) / max(abs(e64), 1e-300)
        errs.append(row)
    out["energy_vs_fp64"] = errs
    for prec in ("mixed", "compensated"):
        ok = [e["a0"] for e in errs if e["rel_err_" + prec] <= 1e-4]
        bad = [e["a0"] for e in errs if e["rel_err_" + prec] > 1e-4]
        out["forms"][prec]["a0_within_1e-4"] = max(ok) if ok else None
        out["forms"][prec]["a0_first_beyond_1e-4"] = min(bad) if bad else None
        out["forms"][prec]["max_rel_energy_err"] = max(e["rel_err_" + prec] for e in errs)
    return out


# --------------------------------------------------------------------------
# Plain-method configuration (Sec. 2.1): 2D 512 x 128 FP64 vacuum, Gaussian
# pulse w0 = 20, sin^2 envelope of ten wavelengths, a0 = 1, one test electron,
# 1000 Boris steps with the Yee and with the customised solver.  4.7 MB of
# state: L2-resident and launch-bound, so no roofline claim is made on it.
# --------------------------------------------------------------------------
def run_c1(stream, steps=1000, oracle_steps=20):
    import torch
    from paper_2004_03754_gb300 import pic as P
    n, dx = (512, 128), (inputs.DX1, inputs.DX2)
    laser = dict(a0=1.0, L_env=20 * np.pi, x_front=336 * dx[0], w0=20.0, x2c=n[1] * dx[1] / 2)
    xe = [np.array([352 * dx[0]]), np.array([n[1] * dx[1] / 2])]
    out = {"workload": "2D 512x128 FP64 vacuum, Gaussian w0=20 a0=1, 10-wavelength sin^2 pulse, "
                       "one test electron, Boris, 1000 steps",
           "l2": "L2-resident (4.7 MB of field state): launch-bound, not a roofline case"}
    for solver in ("yee", "customised"):
        cE, cB = (np.array([1.0]), np.array([1.0])) if solver == "yee" else coeff_table()
        sim = P.Simulation(n, dx, inputs.DT, cE, cB, precision="fp64", pusher="boris",
                           stream=stream.cuda_stream)
        sim.load_laser(**laser)
        sim.load_particles(xe, [np.zeros(1)] * 3, np.zeros(1))
        sim.step(4)
        sim.sync()
        P.pic_set_timing(sim.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t = P.pic_get_timing(sim.ctx)
        sim.close()
        ncell = n[0] * n[1]
        out[solver] = {"ms_per_step": ms / steps, "cell_updates_per_s": ncell * steps / (ms / 1e3),
                       "field_kernel_ms_per_step": t.ms_fields / steps,
                       "field_kernel_gbs_alg": 120.0 * ncell / (t.ms_fields / steps / 1e3) / 1e9,
                       "launches_per_step": t.launches / steps}
    return out


# --------------------------------------------------------------------------
# Differentiation workload: 2D 1024 x 256 vacuum plane wave, a0 = 100, 64 test
# electrons, 4000 Boris steps, checkpoints every 100 steps (FP64)
# --------------------------------------------------------------------------
def run_adjoint(stream):
    from paper_2004_03754_gb300 import pic as P
    cE, cB = coeff_table()
    n = (1024, 256)
    L2 = n[1] * inputs.DX2
    g = inputs.rng(23)
    xs = np.concatenate([(410 + 200 * g.random(64)) * inputs.DX1, g.random(64) * L2])
    us = np.zeros(3 * 64)
    sim = P.Simulation(n, (inputs.DX1, inputs.DX2), inputs.DT, cE, cB, precision="fp64",
                       pusher="boris", stream=stream.cuda_stream)
    las = P.pic_laser(100.0, 1.0, 0.0, 20 * np.pi, 400 * inputs.DX1, 0.0, L2 / 2, 0.0)
    t0 = time.perf_counter()
    J, ga, gp = P.pic_adjoint_laser_energy(sim.ctx, las, xs, us, 4000, 100)
    t_energy = time.perf_counter() - t0
    t0 = time.perf_counter()
    sim.step(4000)
    sim.sync()
    t_fwd = time.perf_counter() - t0
    # broadband vacuum pulse, dispersion objective and its stencil gradient
    x = np.arange(n[0]) * inputs.DX1
    L = n[0] * inputs.DX1
    r = inputs.rng(17)
    modes = range(4, 60, 4)
    amps, phs = r.uniform(0.2, 1.0, len(modes)), r.uniform(0, 2 * np.pi, len(modes))
    f = lambda y: sum(a * np.cos(2 * np.pi * m * y / L + p) for m, a, p in zip(modes, amps, phs))
    e2 = np.tile(f(x), (n[1], 1))
    b3 = np.tile(f(x + inputs.DX1 / 2 + inputs.DT / 2), (n[1], 1))
    tgt = np.tile(f(x - 4000 * inputs.DT), (n[1], 1))
    t0 = time.perf_counter()
    J2, gE, gB = P.pic_adjoint_dispersion(sim.ctx, e2, b3, tgt, 4000, cE.size, 100)
    t_disp = time.perf_counter() - t0
    sim.close()
    Mrow = 2 * np.arange(1, cE.size + 1) - 1.0
    gEp = gE - (gE @ Mrow) / (Mrow @ Mrow) * Mrow
    return {"workload": "2D 1024x256 vacuum plane wave a0=100, 64 test electrons, 4000 steps, "
                        "checkpoint every 100, FP64, Boris",
            "energy": {"J": J, "dJ_da0": ga, "dJ_dphase": gp, "seconds_forward_plus_adjoint": t_energy,
                       "seconds_forward_only": t_fwd},
            "dispersion": {"J": J2, "grad_norm_cE": float(np.linalg.norm(gE)),
                           "grad_norm_cB": float(np.linalg.norm(gB)),
                           "projected_grad_norm_cE": float(np.linalg.norm(gEp)),
                           "seconds_forward_plus_adjoint": t_disp},
            "checked": "tests/test_gpu_adjoint.py: oracle central differences (1e-6) on small "
                       "cases; GPU central differences at this size"}


# --------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# --------------------------------------------------------------------------
def oracle_step_rate(frac=1.0 / 128, seed=inputs.DEFAULT_SEED):
    """Time the oracle on the full field grid: one step without particles and one
    step with each of two random electron samples (frac and 2 frac of the
    workload).  The particle time is fitted as c + a n (c: per-step costs that do
    not grow with n, e.g. the OpenMP build's per-thread current sums) and
    extrapolated to all electrons.  Returns (pushes/s, details)."""
    from oracle import oracle as orc
    cE, cB = coeff_table()
    n, dx, _ = workload_arrays(seed=seed, frac=frac)
    g = orc.Grid(n, dx, inputs.DT, cE, cB)
    F = orc.Fields(g)
    lk = laser_kwargs(n, dx)
    orc.laser_load(g, F, a0=lk["a0"], k0=lk["k0"], phase=lk["phase"], Lenv=lk["L_env"],
                   x_front=lk["x_front"], w0=lk["w0"], x2c=lk["x2c"])
    t0 = time.perf_counter()
    orc.step(g, F, None)
    tf = time.perf_counter() - t0
    pts = []
    for f in (frac, 2 * frac):
        _, _, Ps = workload_arrays(seed=seed, frac=f)
        Po = orc.Particles(Ps.x, Ps.u, Ps.w)
        t0 = time.perf_counter()
        orc.step(g, F, Po)
        pts.append((Ps.n, max(time.perf_counter() - t0 - tf, 1e-9)))
    (n1, t1), (n2, t2) = pts
    a = max((t2 - t1) / (n2 - n1), 1e-12)
    c = max(t1 - a * n1, 0.0)
    n_full = 3585 * 1024 * 8
    t_step_full = tf + c + a * n_full
    return n_full / t_step_full, {"field_s": tf, "particle_sample": n1, "particle_s": t1,
                                  "per_particle_s": a, "fixed_s": c, "t_step_full_s": t_step_full}


def cpu_baseline(args):
    """The FP64 oracle on the host cores: its OpenMP build on every core (the
    reported value) and the plain build on one core."""
    from oracle import oracle as orc
    ncores = os.cpu_count() or 1
    orc.use_openmp(False)
    rate1, det1 = oracle_step_rate()
    orc.use_openmp(True)
    try:
        rate, det = oracle_step_rate()
    finally:
        orc.use_openmp(False)
    sample = ("FP64 oracle steps on the full 4096x1024 grid: without particles, and with "
              "random samples of 1/128 and 1/64 of the electrons (%d, %d); particle time fitted "
              "as fixed + per-particle and extrapolated to all 29,368,320 electrons, plus the "
              "measured field solve" % (det["particle_sample"], 2 * det["particle_sample"]))
    return {"value": rate, "unit": METRIC, "cores": ncores, "kind": "oracle",
            "build": "OpenMP (fields over rows, particles over threads, per-thread currents "
                     "summed in thread order)",
            "sample": sample + " (%.2f s)" % det["field_s"],
            "single_thread": {"value": rate1, "unit": METRIC, "cores": 1,
                              "field_s": det1["field_s"]}}


def c3_leg(stream, steps=8, warmup=3, small=False, fp64=True):
    """3D workload 1024 x 256 x 256 (84,017,152 electrons, a0 = 10, customised
    solver, analytic pusher): ms per step, rates and kernel rooflines for the
    mixed form and the plain FP64 path, for the default bench line."""
    import torch
    from paper_2004_03754_gb300 import pic as P
    n, dx, Pset = c3_workload_arrays(small=small)
    cE, cB = coeff_table()
    peak, peak_kind = measured_peaks()
    ncell = n[0] * n[1] * n[2]
    out = {"workload": "3D %dx%dx%d plasma 2ppc a0=10 w0=30, customised M=16, analytic" % n,
           "particles": Pset.n}
    for precision in (("mixed", "fp64") if fp64 else ("mixed",)):
        k = steps if precision == "mixed" else max(3, steps // 2)
        sim = P.Simulation(n, dx, inputs.DT, cE, cB, precision=precision, pusher="analytic",
                           stream=stream.cuda_stream)
        sim.load_laser(**c3_laser_kwargs(n, dx))
        sim.load_particles(Pset.x, Pset.u, Pset.w, Pset.qm)
        sim.step(warmup)
        sim.sync()
        P.pic_set_timing(sim.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t = P.pic_get_timing(sim.ctx)
        P.pic_set_timing(sim.ctx, False)
        sim.close()
        bpc = 60.0 if precision == "mixed" else 120.0
        fgbs = bpc * ncell / (t.ms_fields / k / 1e3) / 1e9
        pgbs = 104.0 * Pset.n / (t.ms_particles / k / 1e3) / 1e9
        out[precision] = {"ms_per_step": ms / k, "particle_pushes_per_s": Pset.n * k / (ms / 1e3),
                          "cell_updates_per_s": ncell * k / (ms / 1e3),
                          "kernel_ms_per_step": {"rebin": t.ms_rebin / k, "particles": t.ms_particles / k,
                                                 "stragglers": t.ms_stragglers / k,
                                                 "fields": t.ms_fields / k},
                          "field_kernel_roofline": {"bound": "hbm", "achieved": fgbs, "peak": peak,
                                                    "unit": "GB/s", "frac": fgbs / peak,
                                                    "alg_bytes_per_cell": bpc, "peak_kind": peak_kind},
                          "particle_kernel_hbm_view": {"achieved": pgbs, "peak": peak, "unit": "GB/s",
                                                       "frac": pgbs / peak, "alg_bytes_per_push": 104}}
        if precision == "fp64":
            # the FP64 field kernel is bound by the FP64 pipe, not by HBM
            ff = FIELD_FLOP_PER_CELL[3] * ncell / (t.ms_fields / k / 1e3) / 1e12
            out[precision]["field_kernel_roofline"] = {
                "bound": "alu", "achieved": ff, "peak": FP64_PEAK_TFLOPS_AT_MAX,
                "unit": "TFLOP/s (FP64)", "frac": ff / FP64_PEAK_TFLOPS_AT_MAX,
                "alg_flop_per_cell": FIELD_FLOP_PER_CELL[3], "peak_clock_mhz": 2070,
                "hbm_view": {"achieved": fgbs, "peak": peak, "unit": "GB/s", "frac": fgbs / peak,
                             "alg_bytes_per_cell": bpc}}
    if fp64:
        out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


def run_c3(args):
    """3D workload: one JSON line (not the default bench line)."""
    import torch
    from paper_2004_03754_gb300 import pic as P
    n, dx, Pset = c3_workload_arrays(small=args.small)
    cE, cB = coeff_table()
    stream = torch.cuda.Stream()
    out = {"metric": METRIC, "unit": METRIC, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "3D %dx%dx%d plasma 2ppc a0=10 w0=30, customised M=16, analytic" % n,
                      "particles": Pset.n}}
    for precision in (("mixed",) if args.no_fp64 else ("mixed", "fp64")):
        sim = P.Simulation(n, dx, inputs.DT, cE, cB, precision=precision, pusher="analytic",
                           stream=stream.cuda_stream)
        sim.load_laser(**c3_laser_kwargs(n, dx))
        sim.load_particles(Pset.x, Pset.u, Pset.w, Pset.qm)
        sim.step(args.warmup)
        sim.sync()
        P.pic_set_timing(sim.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t = P.pic_get_timing(sim.ctx)
        info = sim.info()
        sim.close()
        k = args.steps
        out[precision] = {"ms_per_step": ms / k, "particle_pushes_per_s": Pset.n * k / (ms / 1e3),
                          "cell_updates_per_s": n[0] * n[1] * n[2] * k / (ms / 1e3),
                          "kernel_ms_per_step": {"rebin": t.ms_rebin / k, "particles": t.ms_particles / k,
                                                 "stragglers": t.ms_stragglers / k, "fields": t.ms_fields / k},
                          "field_gbs": (60.0 if precision == "mixed" else 120.0) * n[0] * n[1] * n[2]
                          / (t.ms_fields / k / 1e3) / 1e9,
                          "sort_interval": info.sort_interval, "tile": list(info.tile)}
    out["value"] = out["mixed"]["particle_pushes_per_s"]
    out["steps"], out["warmup"] = args.steps, args.warmup
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.use_openmp(True)
    vals = []
    for w in range(args.warmup):    # untimed: the same sample steps, other seeds
        oracle_step_rate(frac=1.0 / 2048, seed=inputs.DEFAULT_SEED + 1000 + w)
    t_all = 0.0
    for s in range(args.steps):
        r, det = oracle_step_rate(frac=1.0 / 512, seed=inputs.DEFAULT_SEED + s)
        vals.append(r)
        t_all += det["t_step_full_s"]
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "cells": [4096, 1024],
                                            "particles": 3585 * 1024 * 8, "precision": "fp64"},
            "ms_per_step_kind": "extrapolated: field solve measured on the full grid, particle "
                                "time measured on a 1/512 sample and scaled to all electrons",
            "cpu_baseline": {"value": value, "unit": METRIC, "kind": "oracle",
                             "cores": os.cpu_count() or 1, "build": "OpenMP",
                             "sample": "per step: oracle steps on the full grid without particles "
                                       "and with 1/512 and 1/256 electron samples, extrapolated "
                                       "to all electrons"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--clocks-csv", default=None,
                    help="where the nvidia-smi clock samples of the timed region are written "
                         "(default: one file per local rank in the temporary directory)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-c1", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--small", action="store_true", help="2048x512 cells (profiling size)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3"],
                    help="c2: the 2D bench line (default); c3: the 3D workload, its own line")
    args = ap.parse_args()
    global SMALL, WORKLOAD
    SMALL = args.small
    if SMALL:
        WORKLOAD = WORKLOAD.replace("4096x1024", "2048x512")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c3":
        run_c3(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
