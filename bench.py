#!/usr/bin/env python3
"""Throughput of the explicit electromagnetic PIC hot path on one B300.

One step = the whole hot path for every species: Maxwell half step (E, B,
absorbing edges, laser), current zeroing, sort by tile, the fused gather /
Boris / Esirkepov kernel, Maxwell half step.  The metric is particle-steps
per second of the whole job (alive particles x steps / seconds, summed over
ranks).  The dominant kernel (the fused particle kernel) is also timed by
itself with CUDA events on its own stream, and reported against the measured
HBM copy bandwidth as the roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

--workload selects the set-up (thermal3d, the 3D TSC roofline run, by default;
laser2d, laser3d, thermal2d, heating2d, ensemble, and qed2d, whose steps also
run the nonlinear Compton and Breit-Wheeler passes, reported in a "qed"
object).  The default run adds, on the same line: the FP64 path on the same
workload ("fp64"), the 2D laser-plasma workload ("laser2d"; with FP64 master
fields, "laser2d_fp64_fields"), the issue-rate roof of the fused kernel
("issue_roof"), and in the CPU-baseline leg the
oracle's error on the run's own final state ("oracle_error") and the oracle
timed on all host cores and on one ("cpu_baseline").

Under torchrun each rank runs an independent replica of the workload (the
problems do not exchange data; "scaling": "weak").  --impl reference times
the FP64 CPU oracle on a bounded sample of the same workload on the host's
cores (the particle loop split over threads with private currents).
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
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, pre-steps before warm-up)
    "laser2d": ("2D3V laser-plasma 2048x1024, dx=lambda/32, a0=10 w0=4lambda 8-cycle laser "
                "through an absorbing x-min edge, e-+p slab 10 n_c with 2 lambda ramp, "
                "32+32 particles/cell, TSC, FP32 push + int64 fixed-point deposit", 800),
    "thermal3d": ("3D3V periodic thermal plasma 256^3, 8 electrons/cell (134M), v_th=0.05c, TSC, "
                  "FP32 cell+offset positions, int64 fixed-point deposit", 0),
    "thermal2d": ("2D3V periodic thermal plasma 64x64, 16 electrons/cell, v_th=0.01c, CIC", 0),
    "heating2d": ("2D3V numerical-heating set-up 640x640, dx=lambda/40, e-+ion plasma at 10 n_c, "
                  "kT=1 keV Maxwell-Juttner, 64+64 particles/cell (52M), CIC, periodic, FP32 push + "
                  "int64 fixed-point deposit", 0),
    "laser3d": ("3D3V laser-target 512x256x256, dx=lambda/32, a0=20 w0=2lambda 8-cycle laser through "
                "an absorbing x-min edge, e-+p slab 30 n_c at x in [4,6] lambda, 16+16 particles/cell "
                "(134M), CIC, re-sorted every 10 steps, FP32 push + int64 fixed-point deposit", 400),
    "qed2d": ("2D3V synchrotron cooling of a pair plasma 1024x1024, dx=lambda/32 (0.8 um), e- and e+ "
              "at kT=3000 m c^2 (Maxwell-Juttner), 16+16 particles/cell (33.5M), uniform B_z=4, "
              "nonlinear Compton emission and Breit-Wheeler pair creation passes every step (chi ~ 0.1, "
              "photons pushed at c), TSC, periodic, "
              "FP32 push + int64 fixed-point deposit", 0),
    "ensemble": ("96 independent 2D3V periodic plasmas in one ensemble (batched kernels, persistent "
                 "work-queue particle kernel, one CUDA graph per step): sides 128-768, 4-64 "
                 "particles/cell, v_th 0.005-0.1c, CIC, FP32 + fixed point", 0),
}


def metric_name(workload):
    if workload == "qed2d":
        return ("particle-steps/s (gather+push+deposit, whole step incl. sort, Maxwell and the "
                "nonlinear Compton and Breit-Wheeler passes; photons counted)")
    return "particle-steps/s (gather+push+deposit, whole step incl. sort and Maxwell)"


def make_workload(name, precision, seed_offset=0, ny=None, n3=None, boundary="mur"):
    from paper_2607_13507_b300 import workloads as W
    if name == "laser2d":
        wl = W.laser2d(precision=precision, ny=ny or 1024, boundary=boundary)
    elif name == "thermal3d":
        wl = W.thermal3d(precision=precision, n=n3 or 256)
    elif name == "thermal2d":
        wl = W.thermal2d(precision=precision)
    elif name == "heating2d":
        wl = W.heating2d(res=40, ppc=64, precision=precision)
    elif name == "qed2d":
        wl = W.qed2d(precision=precision, n=ny or 1024)
    elif name == "laser3d":
        wl = W.laser3d(precision=precision, nx=n3 or 512, ny=(n3 or 512) // 2, nz=(n3 or 512) // 2,
                       boundary=boundary)
    else:
        raise SystemExit(f"unknown workload {name}")
    wl.seed += seed_offset
    return wl


def algorithmic_bytes(wl, n_particles, loaded_cells, precision):
    """Bytes the fused kernel must move for one species launch: each particle
    read once and written once, the E/B of the loaded cells read once and the
    current of those cells written once (int64 J, 3 components)."""
    d = wl.dim
    if precision == "fp32":
        rd = 4 + 4 * d + 12 + 4          # cell, offsets, u, w
        wr = 4 + 4 * d + 12              # cell, offsets, u
        grid = 24 + 24                   # E/B float32 read, J int64 written
    else:
        rd = 8 * d + 24 + 8
        wr = 8 * d + 24
        grid = 48 + 24
    return n_particles * (rd + wr) + loaded_cells * grid, rd + wr, grid


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0}, "fallback"


def reduce_over_ranks(elapsed, psteps, device):
    """Replicas (one independent problem per rank, no data-path collective):
    the job's timed region is the longest rank's, its work the sum of the
    ranks' particle-steps."""
    import torch
    import torch.distributed as dist
    mx = torch.tensor([elapsed], dtype=torch.float64, device=device)
    sm = torch.tensor([psteps], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


# the files that define the fused tile kernel k_gpd32 (its code, not its host launcher)
GPD32_SOURCES = ("lpic_common.cuh", "lpic_fp32.cuh", "lpic_qed_tab.cuh", "lpic_gpd32.h", "lpic_gpd32_impl.cuh",
                 "lpic_gpd32_21.cu", "lpic_gpd32_22.cu", "lpic_gpd32_31.cu", "lpic_gpd32_32.cu")


def kernel_source_hash():
    """Hash of the fused kernel's source files: the ncu traffic record is
    valid only for the kernel it was taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2607_13507_b300", "csrc")
    for f in GPD32_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(workload)
    except Exception:
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("bytes_per_launch")


# ------------------------------------------------------------------ the GPU arm
TUNED = os.path.join(ROOT, "paper_2607_13507_b300", "tuned.json")


def tuned_choice(args, wl):
    """Tile shape, particles per block and sort interval: from the command
    line, else from a fresh autotuning run (--autotune), else from the
    committed autotuner results for this workload, else the defaults."""
    from paper_2607_13507_b300 import autotune as A
    ch = {"tile": None, "block_particles": 0, "sort_interval": 0, "source": "defaults"}
    if args.precision != "fp32":
        return ch
    if args.autotune:
        pre = WORKLOADS[args.workload][1] if args.pre_steps is None else args.pre_steps
        best, _ = A.autotune(wl, cache=TUNED if args.autotune_save else None, refresh=True,
                             log=lambda m: print(m, file=sys.stderr), pre_steps=pre)
        ch = {"tile": list(best.tile), "block_particles": best.block_particles,
              "sort_interval": best.sort_interval, "source": "autotune"}
    elif os.path.exists(TUNED):
        rec = json.load(open(TUNED)).get(A.signature(wl))
        if rec:
            c = rec["choice"]
            ch = {"tile": list(c["tile"]), "block_particles": c["block_particles"],
                  "sort_interval": c["sort_interval"], "source": "autotuner results"}
    if ch["source"] == "defaults" and args.workload == "laser3d":
        ch.update(sort_interval=10, source="configuration (re-sort every 10 steps)")
    if args.tile:
        ch.update(tile=[int(v) for v in args.tile.split("x")], source="command line")
    if args.block_particles:
        ch.update(block_particles=args.block_particles, source="command line")
    if args.sort_interval:
        ch.update(sort_interval=args.sort_interval, source="command line")
    return ch

def qed_summary(qed, wl, counts0, counts1, G, peak, which):
    """The QED passes (k_qed_compton32 over each emitting species, then
    k_qed_bw32 over the photons, each followed by a one-thread count clamp)
    timed with CUDA events on the launching stream.
    Algorithmic bytes per emitter per step: cell, offsets, u, id and tau read,
    tau written (8 + 4 dim + 12 B); per photon created: the emitter's weight
    read, its momentum written and the photon written (48 + 4 dim B); the
    fields of the grid read once (24 B per cell).  The pair pass reads each
    photon's cell and momentum (16 B) and, above the pair threshold, its
    offsets, id and depth (not counted)."""
    ms = sum(a.elapsed_time(b) for a, b in qed["events"])
    n_steps = len(qed["events"])
    emit_ids = [i for i, sp in enumerate(G.species) if sp.m > 0]
    ph = G.species.index(qed["photons"])
    n_emit = sum(0.5 * (counts0[i] + counts1[i]) for i in emit_ids)
    created = (counts1[ph] - counts0[ph]) / max(1, n_steps)
    d = wl.dim
    per_emitter = 8 + 4 * d + 12
    per_photon = 48 + 4 * d
    n_ph = 0.5 * (counts0[ph] + counts1[ph])
    bytes_step = n_emit * per_emitter + created * per_photon + 24 * wl.cells + 16 * n_ph
    t = ms / 1e3 / max(1, n_steps)
    if qed["fused"]:
        # the emission runs inside the fused push: its cost is part of the
        # k_gpd32 launch time (the plasma without QED: --qed-mode off)
        return {"kernel": "emission inside k_gpd32 (kGpdQed form) + k_qed_bw32 pass",
                "pair_pass_ms_per_step": 1e3 * t, "emitters": int(n_emit),
                "photons_created_per_step": created, "photons_alive": int(counts1[ph])}
    achieved = bytes_step / t / 1e9
    return {"kernel": "k_qed_compton32 + k_qed_bw32", "ms_per_step": 1e3 * t,
            "emitters": int(n_emit), "photons_created_per_step": created,
            "photons_alive": int(counts1[ph]),
            "emission_passes_per_step": len(emit_ids),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{which} hbm_gbs",
                         "algorithmic_bytes_per_step": bytes_step, "traffic": None}}


def run_b300(args, rank, world, local_rank):
    import torch
    from paper_2607_13507_b300 import build, lpic
    from paper_2607_13507_b300 import workloads as W

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    wl = make_workload(args.workload, args.precision, seed_offset=rank, ny=args.ny, n3=args.n3,
                       boundary=args.boundary)
    prec = lpic.FP32_FIXED if args.precision == "fp32" else lpic.FP64
    tuned = tuned_choice(args, wl)
    parts = W.load_all(wl)
    G = lpic.grid_for(wl, prec, device=dev, tile=tuned["tile"], block_particles=tuned["block_particles"],
                      sort_interval=tuned["sort_interval"], maxwell_fp64=getattr(args, "maxwell_fp64", False))
    for p in parts:
        # a QED set-up keeps room for the pairs created into the lepton species
        cap = (p.n * 9 // 8 + 63) // 64 * 64 if wl.qed_eps_ref > 0 else None
        G.add_species(p, capacity=cap, stream=stream)
    loaded = [p.n // wl.species[i].ppc for i, p in enumerate(parts)]
    qed = None
    if wl.qed_eps_ref > 0 and args.qed_mode == "off":
        # the same plasma without QED (the baseline of the QED cost)
        wl.qed_eps_ref = 0.0
        G.B[2].fill_(wl.b0)
    if wl.qed_eps_ref > 0:
        # photons appended by the emission passes; depths indexed by the
        # (species-unique) particle ids
        n_ids = sum(p.n for p in parts)
        phot = G.add_empty_species(0.0, 0.0, n_ids // 2, stream=stream)
        G.B[2].fill_(wl.b0)
        G.qed_init(wl.qed_eps_ref, wl.seed, stream)
        emitters = [sp for sp in G.species if sp.m > 0]
        # ids of the particles created later: a range of their own per species
        # (the depths and the random draws are keyed by id)
        n_tau = n_ids
        for sp in emitters:
            sp.set_next_id(n_tau, stream)
            n_tau += sp.cap
        qed = dict(emitters=emitters, photons=phot, tau=G.qed_initial_tau(n_tau, stream),
                   ph_tau=torch.zeros(phot.cap, dtype=torch.float32, device=dev), events=[],
                   pairs=(emitters[0], emitters[1]) if len(emitters) == 2 else None,
                   fused=args.qed_mode == "fused")
        if qed["fused"]:
            # emission inside the fused push of each lepton species (Algorithm 1)
            for sp in emitters:
                G.qed_fuse(sp, phot, qed["tau"], first_step=0, stream=stream, photon_tau=qed["ph_tau"])
    del parts
    dt = G.dt
    pre = WORKLOADS[args.workload][1] if args.pre_steps is None else args.pre_steps

    def advance(k, timed=False):
        """One step of the path (and the emission passes of a QED workload)."""
        G.step(k * dt, stream)
        if qed is None:
            return
        if timed:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
        if not qed["fused"]:
            for sp in qed["emitters"]:
                G.qed_compton(sp, qed["photons"], qed["tau"], k, stream, photon_tau=qed["ph_tau"])
        if qed["pairs"] is not None:
            G.qed_breit_wheeler(qed["photons"], *qed["pairs"], qed["ph_tau"], k, stream)
        if timed:
            ev[1].record(stream)
            qed["events"].append(ev)

    step = 0
    with torch.cuda.stream(stream):
        for _ in range(pre + args.warmup):
            advance(step)
            step += 1
    stream.synchronize()
    if G.check_status(stream) != 0:
        raise SystemExit("device status bits set during warm-up")
    counts0 = [sp.query(stream)[1] for sp in G.species]

    if world > 1:
        torch.distributed.barrier()
    clock = ClockSampler(local_rank)
    clock.start()
    time.sleep(0.3)
    launches0 = G.info().launches
    unfused = bool(getattr(args, "unfused", False))
    if unfused and qed is not None:
        raise SystemExit("--unfused does not apply to the QED workload")
    bufs = [torch.empty((6, sp.cap), dtype=torch.float32, device=dev) for sp in G.species] if unfused else []

    def one_step(t):
        if not unfused:
            advance(step, timed=True)
            return
        # the unfused path: gather stage, (hooks would go here), push/deposit stage
        G.maxwell_half(0, t, stream)
        G.zero_current(stream)
        for sid in range(len(G.species)):
            G.gather_fields(sid, out=bufs[sid], stream=stream)
            G.push_deposit_fields(sid, bufs[sid], stream=stream)
        G.maxwell_half(1, t + 0.5 * dt, stream)

    G.kernel_timing(args.steps * len(G.species) * (2 if unfused else 1))
    t_start, t_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            one_step(step * dt)
            step += 1
    t_stop.record(stream)
    torch.cuda.synchronize(dev)
    elapsed = t_start.elapsed_time(t_stop) / 1e3
    launches = G.info().launches - launches0
    clocks = clock.stop()
    if G.check_status(stream) != 0:
        raise SystemExit("device status bits set during the timed steps")
    counts1 = [sp.query(stream)[1] for sp in G.species]
    psteps = sum(0.5 * (a + b) for a, b in zip(counts0, counts1)) * args.steps

    # dominant kernel: per-launch times (events recorded by the library on the
    # kernel's stream) and algorithmic bytes
    gpd_ms, gpd_launches = G.kernel_time()
    G.kernel_timing(0)
    gpd_time = gpd_ms / 1e3
    algo_bytes_step = 0
    massive = [i for i, sp in enumerate(G.species) if sp.m > 0]      # photons skip the fused kernel
    for i in massive:
        n_mean = 0.5 * (counts0[i] + counts1[i])
        algo_bytes_step += algorithmic_bytes(wl, n_mean, loaded[i], args.precision)[0]
    launch_bytes = algo_bytes_step / len(massive)
    launch_time = gpd_time / max(1, gpd_launches)
    if unfused:
        # a "launch" is the pair of stages; the field array adds 24 B written
        # and 24 B read per particle
        n_mean_all = sum(0.5 * (a + b) for a, b in zip(counts0, counts1))
        launch_bytes += 48.0 * n_mean_all / len(G.species)
        launch_time *= 2.0

    if world > 1:
        elapsed, psteps = reduce_over_ranks(elapsed, psteps, dev)

    result = None
    if rank == 0:
        peaks, which = measured_peaks()
        peak = float(peaks["hbm_gbs"])
        achieved = launch_bytes / launch_time / 1e9
        per_ps = algorithmic_bytes(wl, 1, 0, args.precision)[1]
        result = {
            "metric": metric_name(args.workload),
            "value": psteps / elapsed,
            "unit": "particle-steps/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f32 (int64 fixed-point current" + (", f64 fields)" if getattr(args, "maxwell_fp64", False)
                                                          else ")")) if args.precision == "fp32" else "f64",
            "data": "synthetic (seeded Philox initial conditions)",
            "config": {
                "workload": WORKLOADS[args.workload][0] + (
                    "; CPML x layers of 16 cells, laser entering as a current sheet"
                    if args.boundary == "cpml" else "") + (
                    "; unfused path (gather stage, then push/deposit stage)" if unfused else ""),
                "grid": list(wl.n), "species": len(wl.species),
                "particles": int(sum(counts0)), "pre_steps": pre,
                "l2": "inputs larger than L2 (particle state %.1f GB)" % (
                    sum(counts0) * algorithmic_bytes(wl, 1, 0, args.precision)[1] / 2 / 1e9),
                "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            },
            "gpd_particle_steps_per_s": psteps / max(gpd_time, 1e-12) if world == 1 else None,
            "roofline": {
                "bound": "hbm",
                "kernel": ("k_gpd32 gather + fields-in stages" if unfused else "k_gpd32")
                if args.precision == "fp32" else "k_gpd64",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{which} hbm_gbs",
                "bytes_per_particle_step": per_ps + (48 if unfused else 0),
                "algorithmic_bytes_per_launch": launch_bytes,
                "launch_ms": 1e3 * launch_time,
                "traffic": None if unfused else ncu_traffic(args.workload),
            },
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        if qed is not None:
            result["qed"] = qed_summary(qed, wl, counts0, counts1, G, peak, which)
    if result is not None:
        result["config"]["tuning"] = tuned
    state = dict(G=G, stream=stream, dev=dev, step=step, counts=counts1, wl=wl, advance=advance,
                 extra=[qed["tau"], qed["ph_tau"]] if qed is not None else [])
    return result, state


def run_ensemble(args, rank, world, local_rank):
    """The batched ensemble: every step of all members is one replay of the
    captured ensemble step (batched field and sort kernels, one persistent
    particle kernel over the device work queue)."""
    import torch
    from paper_2607_13507_b300 import build, lpic
    from paper_2607_13507_b300 import workloads as W
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    members = W.ensemble(count=args.ensemble_count, seed=W.SEED_BASE + 4000 + 97 * rank)
    if args.ensemble_tuning == "per-member":
        from paper_2607_13507_b300 import autotune as AT
        choices, classes = AT.tune_ensemble(members, cache=os.path.join(ROOT, "paper_2607_13507_b300",
                                                                        "tuned.json"))
        tuning = {"rule": "per member: the best (tile, block_particles) of its particles-per-cell class, "
                          "each class timed alone on a 512x512 periodic plasma (autotuner results)",
                  "classes": {str(c): {"tile": list(v[0].tile), "block_particles": v[0].block_particles}
                              for c, v in classes.items()}}
    else:
        from paper_2607_13507_b300.autotune import Choice
        choices = [Choice((16, 8), 0, 1)] * len(members)
        tuning = {"rule": "uniform", "tile": [16, 8]}
    grids, counts, loaded = [], 0, 0
    for wl, ch in zip(members, choices):
        parts = W.load_all(wl)
        G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=ch.tile, device=dev, block_particles=ch.block_particles)
        G.add_species(parts[0], stream=stream)
        counts += parts[0].n
        loaded += parts[0].n // wl.species[0].ppc
        grids.append(G)
        del parts
    ens = lpic.Ensemble(grids)
    ens.graph_steps(args.warmup, stream)
    stream.synchronize()
    if ens.check_status(stream) != 0:
        raise SystemExit("device status bits set during warm-up")
    if world > 1:
        torch.distributed.barrier()
    clock = ClockSampler(local_rank)
    clock.start()
    time.sleep(0.3)
    l0 = ens.launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(stream)
    ens.graph_steps(args.steps, stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    elapsed = a.elapsed_time(b) / 1e3
    clocks = clock.stop()
    if ens.check_status(stream) != 0:
        raise SystemExit("device status bits set during the timed steps")
    n_now = sum(G.species[0].query(stream)[1] for G in grids)
    psteps = 0.5 * (counts + n_now) * args.steps
    if world > 1:
        elapsed, psteps = reduce_over_ranks(elapsed, psteps, dev)
    if rank != 0:
        return None
    peaks, which = measured_peaks()
    wl0 = members[0]
    per_ps = algorithmic_bytes(wl0, 1, 0, "fp32")[1]
    step_bytes = counts * per_ps + loaded * algorithmic_bytes(wl0, 0, 1, "fp32")[2]
    achieved = step_bytes / (elapsed / args.steps) / 1e9
    return {
        "metric": metric_name(args.workload),
        "value": psteps / elapsed, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (int64 fixed-point current)",
        "data": "synthetic (seeded Philox initial conditions)",
        "config": {"workload": WORKLOADS["ensemble"][0], "members": len(members),
                   "particles": int(counts), "l2": "inputs larger than L2", "tuning": tuning,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "whole ensemble step", "achieved": achieved,
                     "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                     "frac": achieved / float(peaks["hbm_gbs"]), "peak_source": f"{which} hbm_gbs",
                     "traffic": None},
        "gpu_launches": int(ens.launches() - l0), "clocks": clocks,
    }


def run_e2e(args, st):
    """Same metric through host buffers: every step copies the state (particle
    buffers and fields) from pinned host memory to the device, runs the step,
    and copies the state back to pinned host memory."""
    import torch
    G, stream, dev = st["G"], st["stream"], st["dev"]
    dt = G.dt
    cur = [sp.query(stream)[0] for sp in G.species]
    host_p = [torch.empty(sp.buffers[0].shape, dtype=sp.buffers[0].dtype, pin_memory=True)
              for sp in G.species]
    for h, sp, c in zip(host_p, G.species, cur):
        h.copy_(sp.buffers[c])
    fields = G.E + G.B + G.J + st["extra"]
    host_f = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in fields]
    for h, f in zip(host_f, fields):
        h.copy_(f)
    nbytes = sum(h.numel() * h.element_size() for h in host_p + host_f)
    steps = max(1, min(args.steps, args.e2e_steps))
    step = st["step"]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    psteps = 0
    with torch.cuda.stream(stream):
        for _ in range(steps):
            for h, sp, c in zip(host_p, G.species, cur):
                sp.buffers[c].copy_(h, non_blocking=True)
            for h, f in zip(host_f, fields):
                f.copy_(h, non_blocking=True)
            st["advance"](step)
            step += 1
            for i, sp in enumerate(G.species):
                cur[i], n = sp.query(stream)
                psteps += n
                host_p[i].copy_(sp.buffers[cur[i]], non_blocking=True)
            for h, f in zip(host_f, fields):
                h.copy_(f, non_blocking=True)
            stream.synchronize()
    el = time.perf_counter() - t0
    return {"value": psteps / el, "unit": "particle-steps/s", "h2d_bytes_per_step": int(nbytes),
            "d2h_bytes_per_step": int(nbytes), "steps": steps}


# ------------------------------------------------------------------ the oracle
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class _ThreadedOracleStep:
    """One step of the FP64 oracle with its particle loop split over threads:
    the unchanged oracle functions (Yee half steps, per-species push with
    gather, Boris and Esirkepov deposit) called on per-thread slices of the
    particles, each slice depositing into a private current array that shares
    the grid's E and B; the private currents are summed before the second
    half step (the OpenMP-over-patches scheme of Sec. 2.3, with threads in
    place of patches).  The oracle releases the interpreter lock while it
    runs, so the slices run concurrently."""

    def __init__(self, O, g, species, threads):
        import numpy as np
        from concurrent.futures import ThreadPoolExecutor
        self.O, self.g, self.threads = O, g, max(1, int(threads))
        self.jobs = []
        self.grids = []
        for k in range(self.threads):
            gk = O.Grid(g.dim, (g.nx, g.ny, g.nz)[:g.dim], (g.dx, g.dy, g.dz)[:g.dim], g.dt, g.order,
                        absorb_x=g.absorb_x)
            gk.E, gk.B = g.E, g.B
            self.grids.append(gk)
        for sp in species:
            cuts = np.linspace(0, sp.n, self.threads + 1).astype(np.int64)
            for k in range(self.threads):
                a, b = int(cuts[k]), int(cuts[k + 1])
                if b > a:
                    part = O.Species(sp.q, sp.m, sp.x[:g.dim, a:b], sp.u[:, a:b], sp.w[a:b],
                                     alive=sp.alive[a:b])
                    self.jobs.append((k, part))
        self.pool = ThreadPoolExecutor(max_workers=self.threads) if self.threads > 1 else None

    def alive(self):
        return sum(int(part.alive.sum()) for _, part in self.jobs)

    def __call__(self, t):
        O, g = self.O, self.g
        O.maxwell_half(g, 0, t)
        for gk in self.grids:
            for c in range(3):
                gk.J[c][...] = 0.0

        def run(k):
            for kk, part in self.jobs:
                if kk == k:
                    O.push_species(self.grids[k], part)

        if self.pool is None:
            run(0)
        else:
            list(self.pool.map(run, range(self.threads)))
        for c in range(3):
            g.J[c][...] = sum(gk.J[c] for gk in self.grids)
        O.maxwell_half(g, 1, t + 0.5 * g.dt)


def oracle_sample(args, budget_s, max_steps, threads=1):
    """Time the FP64 CPU oracle on a bounded sample of the workload: the full
    x extent with the first 16 rows (2D), the full x extent with 8 x 8 cells
    across (3D laser-target: the slab lies along x) or a 32^3 box (3D
    thermal), same cell size, density profile and particles per cell.  With
    threads > 1 the particle loop runs on that many host threads (private
    currents, summed); the QED set-up runs on one thread."""
    import numpy as np
    from oracle import oracle as O
    from paper_2607_13507_b300 import workloads as W
    wl = make_workload(args.workload, "fp64", boundary=args.boundary)
    if wl.qed_eps_ref > 0:
        # the oracle's emission rate integrates the spectrum afresh for every
        # particle (about 0.07 s each): a 4 x 4-cell box
        sample = dict(n=(4, 4))
        threads = 1
    elif wl.dim == 2:
        sample = dict(n=(wl.n[0], min(16, wl.n[1])))
    elif wl.laser is not None:
        sample = dict(n=(wl.n[0], 8, 8))
    else:
        sample = dict(n=(32, 32, 32))
    wl.n = sample["n"]
    parts = W.load_all(wl)
    laser = None
    if wl.laser is not None:
        c = wl.laser_center()
        laser = O.Laser(wl.laser.a0, wl.laser.w0, wl.laser.tau, wl.laser.omega, c[0],
                        c[1] if wl.dim == 3 else 0.0)
    pml = O.Pml() if wl.boundary == "cpml" else None
    g = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=wl.absorb_x, laser=laser, pml=pml)
    h = np.array(wl.h)[:, None]
    sps = [O.Species(p.q, p.m, (p.cell + p.off) * h, p.u, p.w) for p in parts]
    npart = sum(p.n for p in parts)
    tau = None
    if wl.qed_eps_ref > 0:
        g.B[2][...] = wl.b0
    if wl.qed_eps_ref > 0 and getattr(args, "qed_mode", "fused") != "off":
        ids = np.concatenate([p.id for p in parts])
        tau = [O.qed_initial_tau(p.id, wl.seed) for p in parts]
        assert len(set(ids.tolist())) == len(ids)
    stepper = _ThreadedOracleStep(O, g, sps, threads) if (threads > 1 and tau is None and pml is None) else None
    if stepper is None:
        threads = 1
    phots = []
    nemit = len(sps)
    t0 = time.perf_counter()
    steps = 0
    psteps = 0
    while steps < max_steps and (time.perf_counter() - t0) < budget_s:
        if stepper is not None:
            psteps += stepper.alive()
            stepper(steps * wl.dt)
            steps += 1
            continue
        psteps += sum(int(sp.alive.sum()) for sp in sps)
        if tau is not None and getattr(args, "qed_mode", "fused") == "fused":
            # emission inside the particle loop (Algorithm 1)
            t = steps * wl.dt
            O.maxwell_half(g, 0, t)
            for c in range(3):
                g.J[c][...] = 0.0
            new = []
            for k, sp in enumerate(list(sps)):
                if k < nemit:
                    ph, _ = O.push_species_qed(g, sp, wl.qed_eps_ref, wl.seed, steps, tau[k])
                    if ph.x.shape[1]:
                        new.append(ph)
                else:
                    O.push_species(g, sp)
            O.maxwell_half(g, 1, t + 0.5 * wl.dt)
            for ph in new:
                sps.append(ph)
                phots.append((ph, O.qed_initial_tau_kind(np.arange(ph.x.shape[1]), 3, wl.seed)))
            for ph, pt in list(phots):                   # pair creation by the photons
                e_, p_ = O.qed_bw(g, ph, wl.qed_eps_ref, wl.seed, steps, pt)
                sps += [s for s in (e_, p_) if s.x.shape[1]]
            steps += 1
            continue
        O.step(g, sps, steps * wl.dt)
        if tau is not None:
            for k in range(nemit):
                ph = O.qed_compton(g, sps[k], wl.qed_eps_ref, wl.seed, steps, tau[k])
                if ph.x.shape[1]:
                    sps.append(ph)
                    phots.append((ph, O.qed_initial_tau_kind(np.arange(ph.x.shape[1]), 3, wl.seed)))
            for ph, pt in list(phots):                   # pair creation by the photons
                e_, p_ = O.qed_bw(g, ph, wl.qed_eps_ref, wl.seed, steps, pt)
                sps += [s for s in (e_, p_) if s.x.shape[1]]
        steps += 1
    el = time.perf_counter() - t0
    desc = (f"{'x'.join(str(v) for v in wl.n)} cells of the workload (same dx, profile, ppc), "
            f"{npart} particles, {steps} steps, FP64 oracle, {threads} thread{'s' if threads > 1 else ''}")
    return psteps / el, desc, steps, el, threads


def oracle_error(state, n_sample=2000):
    """The run's own final state against the oracle: 2000 particles drawn at
    random are pushed by the FP64 oracle in the GPU's own (float) fields and
    compared with the GPU's push of the same step (momenta relative to |u|,
    positions in cells at the integer time), and the integer continuity
    residual rho1 - rho0 + div J of that step over the whole grid (periodic
    grids; interior columns with absorbing x), which the fixed-point deposit
    makes exactly zero."""
    import numpy as np
    import torch
    from oracle import oracle as O
    G, stream, wl = state["G"], state["stream"], state["wl"]
    if G.precision != 1:
        return None
    t = state["step"] * wl.dt
    G.maxwell_half(0, t, stream)
    G.zero_current(stream)
    sp = max(G.species, key=lambda s: s.query(stream)[1])
    G.sort(sp.id, stream)
    st = sp.state(stream)
    n = st["id"].shape[0]
    rng = np.random.Generator(np.random.Philox(20261204))
    pick = rng.choice(n, size=min(n_sample, n), replace=False)
    ids = st["id"][pick]
    rho0 = sp.charge(stream)
    g = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=wl.absorb_x)
    for c in range(3):
        g.E[c][...] = G.E[c].cpu().numpy().astype(np.float64)
        g.B[c][...] = G.B[c].cpu().numpy().astype(np.float64)
    h = np.array(wl.h)[:, None]
    u = st["u"][:, pick].astype(np.float64)
    gam = np.sqrt(1.0 + (u ** 2).sum(0))
    cell = st["cell"][pick].astype(np.int64)
    coords = [cell % wl.n[0], (cell // wl.n[0]) % wl.n[1]]
    if wl.dim == 3:
        coords.append(cell // (wl.n[0] * wl.n[1]))
    x_half = (np.stack(coords).astype(np.float64) + st["off"][:, pick].astype(np.float64)) * h
    x_int = x_half - 0.5 * wl.dt * u[:wl.dim] / gam
    osp = O.Species(sp.q, sp.m, x_int, u, st["w"][pick].astype(np.float64))
    O.push_species(g, osp)
    G.gather_push_deposit(sp.id, stream)
    torch.cuda.synchronize()
    st1 = sp.state(stream)
    x1 = sp.positions_at_step(stream)
    order = np.argsort(st1["id"])
    pos = np.searchsorted(st1["id"][order], ids)
    pos = np.clip(pos, 0, len(order) - 1)
    rows = order[pos]
    keep = (st1["id"][rows] == ids) & (osp.alive != 0)
    ug = st1["u"][:, rows[keep]].astype(np.float64)
    uo = osp.u[:, keep]
    rel_u = float(np.max(np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-30)))
    diff = x1[:, rows[keep]] - osp.x[:wl.dim, keep]
    L = np.array(wl.n)[:, None] * h
    for d in range(wl.dim):
        if d > 0 or not wl.absorb_x:
            diff[d] = np.remainder(diff[d] + 0.5 * L[d], L[d]) - 0.5 * L[d]
    dx = float(np.max(np.abs(diff) / h))
    rho1 = sp.charge(stream)
    J = G.J
    div = (J[0] - torch.roll(J[0], 1, -1)) + (J[1] - torch.roll(J[1], 1, -2))
    if wl.dim == 3:
        div = div + (J[2] - torch.roll(J[2], 1, -3))
    res = rho1 - rho0 + div
    if wl.absorb_x:
        res = res[..., 4:-4]
    return {"species": "the most populous species", "sampled_particles": int(keep.sum()),
            "momentum_rel_max": rel_u, "position_cells_max": dx,
            "continuity_nonzero_nodes": int(torch.count_nonzero(res).item()),
            "continuity_nodes": int(res.numel()),
            "reference": "FP64 oracle push of the sample in the GPU's fields, same step"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    val, desc, steps, el, used = oracle_sample(args, budget_s=max(10.0, 0.5 * (args.steps + args.warmup)),
                                               max_steps=args.steps + args.warmup, threads=host_cores())
    return {
        "metric": metric_name(args.workload),
        "value": val, "unit": "particle-steps/s", "n_gpus": world, "steps": steps,
        "warmup": 0, "ms_per_step": 1e3 * el / max(steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Philox initial conditions)",
        "config": {"workload": WORKLOADS[args.workload][0], "sample": desc},
        "impl": "reference",
        "cpu_baseline": {"value": val, "unit": "particle-steps/s", "cores": used, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": val, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def issue_roof(res, workload, clocks):
    """The fused kernel against the instruction-issue roof: warp instructions
    per particle from the committed ncu capture of the same kernel source
    (profiles/issue.json) times the measured particle rate of the kernel,
    over SMs x 4 schedulers x the median SM clock seen in the timed region."""
    path = os.path.join(ROOT, "profiles", "issue.json")
    try:
        rec = json.load(open(path)).get(workload)
    except Exception:
        rec = None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2032.0
    rate = res.get("gpd_particle_steps_per_s")
    if not rate:
        return None
    achieved = rec["warp_inst_per_particle"] * rate
    peak = nsm * 4 * mhz * 1e6
    return {"warp_inst_per_particle": rec["warp_inst_per_particle"], "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak, "captured": rec.get("captured")}


def side_line(args, workload, precision, steps, warmup, maxwell_fp64=False):
    """The same contract's numbers for another workload or precision, run in
    this process after the main line (no e2e, no baseline)."""
    import copy
    import torch
    sub = copy.copy(args)
    sub.workload, sub.precision, sub.steps, sub.warmup = workload, precision, steps, warmup
    sub.maxwell_fp64 = maxwell_fp64
    sub.pre_steps = None
    sub.tile, sub.block_particles, sub.sort_interval = None, 0, 0
    res, state = run_b300(sub, 0, 1, 0)
    del state
    torch.cuda.empty_cache()
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "gpd_particle_steps_per_s", "clocks")
    out = {k: res[k] for k in keep if k in res}
    out["workload"] = res["config"]["workload"]
    out["particles"] = res["config"]["particles"]
    r = res["roofline"]
    out["roofline"] = {k: r[k] for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "peak_source",
                                         "bytes_per_particle_step", "launch_ms", "traffic")}
    if precision == "fp32":
        out["config"] = {"tuning": res["config"].get("tuning")}
        out["issue_roof"] = issue_roof(res, workload, res.get("clocks"))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["b300", "reference"], default="b300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="thermal3d")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--pre-steps", type=int, default=None,
                    help="untimed steps before warm-up (default: bring the laser onto the target)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ensemble-count", type=int, default=96)
    ap.add_argument("--qed-mode", choices=("fused", "passes", "off"), default="fused",
                    help="qed2d: emission inside the fused push (Algorithm 1), as separate passes after "
                         "the step, or no QED (the same plasma)")
    ap.add_argument("--ensemble-tuning", choices=("per-member", "uniform"), default="per-member",
                    help="ensemble launch choices: per particles-per-cell class (autotuned) or one (16, 8) tile")
    ap.add_argument("--tile", default=None, help="tile shape, e.g. 8x8")
    ap.add_argument("--block-particles", type=int, default=0)
    ap.add_argument("--sort-interval", type=int, default=0)
    ap.add_argument("--autotune", action="store_true", help="autotune tile/block/sort interval first")
    ap.add_argument("--autotune-save", action="store_true", help="store the autotuner result")
    ap.add_argument("--n3", type=int, default=None,
                    help="cells per side of the 3D thermal workload (smaller cases for profiling)")
    ap.add_argument("--ny", type=int, default=None,
                    help="transverse cells of the 2D laser workload (smaller cases for profiling)")
    ap.add_argument("--boundary", choices=["mur", "cpml"], default="mur",
                    help="absorbing x of the laser workloads: Mur edges or CPML layers")
    ap.add_argument("--unfused", action="store_true",
                    help="time the unfused path (gather stage + push/deposit stage) instead of the fused kernel")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the FP64 and 2D laser-plasma lines of the default run")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--maxwell-fp64", action="store_true",
                    help="FP32 particles with FP64 master fields (Maxwell half steps in double)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return

    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.workload == "ensemble":
        res = run_ensemble(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    res, state = run_b300(args, rank, world, local_rank)
    if rank == 0:
        if args.precision == "fp32" and not args.unfused:
            res["issue_roof"] = issue_roof(res, args.workload, res.get("clocks"))
        if not args.no_e2e:
            res["e2e"] = run_e2e(args, state)
        leg = None
        if world == 1 and not args.no_cpu_baseline:
            # the oracle's error on this run's state, before the state goes
            leg = {"oracle_error": oracle_error(state)} if args.precision == "fp32" and not args.unfused else {}
        del state
        torch.cuda.empty_cache()
        default_run = (args.workload == "thermal3d" and args.n3 is None and args.precision == "fp32"
                       and world == 1 and not args.no_side and not args.unfused)
        if default_run:
            res["fp64"] = side_line(args, "thermal3d", "fp64", args.fp64_steps, 3)
            res["laser2d"] = side_line(args, "laser2d", "fp32", 20, 3)
            res["laser2d_fp64_fields"] = side_line(args, "laser2d", "fp32", 20, 3, maxwell_fp64=True)
        if leg is not None:
            n = host_cores()
            val, desc, steps, el, used = oracle_sample(args, args.cpu_budget, 60, threads=n)
            v1, d1, s1, e1, _ = oracle_sample(args, args.cpu_budget, 60, threads=1)
            res["cpu_baseline"] = {"value": val, "unit": "particle-steps/s", "cores": used, "nproc": n,
                                   "kind": "oracle", "sample": desc,
                                   "one_core": {"value": v1, "unit": "particle-steps/s", "cores": 1,
                                                "sample": d1}}
            if "oracle_error" in leg:
                res["oracle_error"] = leg["oracle_error"]
        print(json.dumps(res), flush=True)
    else:
        del state
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
