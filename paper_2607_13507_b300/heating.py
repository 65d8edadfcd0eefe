"""Numerical-heating study (Sec. 4.1) on the GPU path.

A uniform 2D electron-ion plasma (n_e = 10 n_c, kT = 1 keV Maxwell-Juttner
momenta for both species, periodic, cloud-in-cell shapes, dt = 0.95 CFL) is
evolved for 5000 / omega_pe while the total energy (kinetic + field, FP64
reductions on the device) is recorded every 10 steps; the study reports the
drift dE/E0 = (E_kin + E_field - E0) / E0 for dx = lambda/20 and lambda/40 and
16 and 64 particles per cell and species.

    python -m paper_2607_13507_b300.heating [--precision fp32|fp64]
        [--res 20 40] [--ppc 16 64] [--box 16] [--fraction 1.0] [--out file.json]

The steps between two records run as replays of a captured CUDA graph.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import torch

from . import lpic
from . import workloads as W


def run(res: int, ppc: int, precision: str = "fp32", box: float = 16.0, fraction: float = 1.0,
        every: int = 10, device: str = "cuda") -> dict:
    wl = W.heating2d(res=res, ppc=ppc, L_lambda=box, precision=precision)
    prec = lpic.FP32_FIXED if precision == "fp32" else lpic.FP64
    stream = torch.cuda.Stream(device=device)
    G = lpic.grid_for(wl, prec, device=device)
    parts = W.load_all(wl)
    for p in parts:
        G.add_species(p, stream=stream)
    npart = sum(p.n for p in parts)
    del parts
    steps = int(math.ceil(fraction * wl.steps / every)) * every
    G.set_clock(0.0, stream)
    hist = []
    t0 = time.perf_counter()
    e0 = None
    for k in range(steps // every + 1):
        d = G.diagnostics(stream)
        e = d.kinetic + d.field
        e0 = e if e0 is None else e0
        hist.append((k * every * wl.dt * math.sqrt(10.0), (e - e0) / e0))
        if k < steps // every:
            G.graph_steps(every, stream)
    stream.synchronize()
    el = time.perf_counter() - t0
    if G.check_status(stream) != 0:
        raise RuntimeError("device status bits set during the heating run")
    return {"config": wl.name, "dx": f"lambda/{res}", "ppc": ppc, "cells": list(wl.n),
            "particles": npart, "steps": steps, "dt": wl.dt, "precision": precision,
            "t_end_wpe": hist[-1][0], "dE_over_E0_end": hist[-1][1],
            "dE_over_E0_max": max(abs(h[1]) for h in hist), "wall_s": el,
            "history_every_10_steps": [[round(t, 4), h] for t, h in hist]}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--res", type=int, nargs="+", default=[20, 40])
    ap.add_argument("--ppc", type=int, nargs="+", default=[16, 64])
    ap.add_argument("--box", type=float, default=16.0, help="box side in laser wavelengths")
    ap.add_argument("--fraction", type=float, default=1.0, help="fraction of 5000 / omega_pe to run")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = []
    for r in a.res:
        for p in a.ppc:
            out = run(r, p, a.precision, a.box, a.fraction)
            res.append(out)
            short = {k: v for k, v in out.items() if k != "history_every_10_steps"}
            print(json.dumps(short), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)
    return res


if __name__ == "__main__":
    main(sys.argv[1:])
