"""Autotuner for the FP32 path: tile shape, particles per thread block and
sort interval.

Each candidate is timed on the actual workload for a few full steps
(CUDA events on the stepping stream, after warm-up); the fastest wins.  The
search is staged to keep it short: tile shape x sort interval at the default
block size, then the block size for the best pair.  Results can be cached in
a JSON file keyed by the workload's signature (grid, cell sizes, shape order,
species, particles per cell, boundaries).
"""
from __future__ import annotations

import itertools
import json
import os
from dataclasses import asdict, dataclass

import torch

from . import lpic
from . import workloads as W


@dataclass(frozen=True)
class Choice:
    tile: tuple
    block_particles: int
    sort_interval: int


def signature(wl: W.Workload) -> str:
    sp = ";".join(f"{s.q},{s.m},{s.ppc},{s.profile}" for s in wl.species)
    return f"{wl.dim}|{wl.n}|{tuple(round(h, 9) for h in wl.h)}|{wl.order}|{int(wl.absorb_x)}|{sp}"


def default_tiles(dim: int, n: tuple) -> list:
    if dim == 2:
        cands = [(8, 8), (16, 8), (16, 16), (32, 8)]
    else:
        cands = [(8, 8, 8), (8, 8, 4), (4, 4, 4)]
    return [t for t in cands if all(t[d] <= n[d] for d in range(dim))]


def time_choice(wl, parts, ch: Choice, steps=6, warmup=2, stream=None, device="cuda") -> float:
    """Milliseconds per full step of the workload with this choice."""
    st = stream or torch.cuda.current_stream()
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=ch.tile, device=device,
                      block_particles=ch.block_particles, sort_interval=ch.sort_interval)
    try:
        for p in parts:
            G.add_species(p, stream=st)
        for s in range(warmup):
            G.step(s * G.dt, st)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.synchronize()
        a.record(st)
        for s in range(warmup, warmup + steps):
            G.step(s * G.dt, st)
        b.record(st)
        st.synchronize()
        if G.check_status(st) != 0:
            return float("inf")
        return a.elapsed_time(b) / steps
    finally:
        G.close()
        del G
        torch.cuda.empty_cache()


def autotune(wl: W.Workload, tiles=None, intervals=(1, 2, 3), block_sizes=(2048, 4096, 8192),
             steps=6, warmup=2, cache: str | None = None, log=None) -> tuple:
    """Returns (best Choice, list of (Choice, ms per step))."""
    key = signature(wl)
    if cache and os.path.exists(cache):
        try:
            rec = json.load(open(cache)).get(key)
            if rec:
                c = rec["choice"]
                return Choice(tuple(c["tile"]), c["block_particles"], c["sort_interval"]), rec["table"]
        except (OSError, ValueError, KeyError):
            pass
    parts = W.load_all(wl)
    stream = torch.cuda.Stream()
    table = []

    def measure(ch):
        ms = time_choice(wl, parts, ch, steps, warmup, stream)
        table.append((ch, ms))
        if log:
            log(f"autotune {ch} -> {ms:.3f} ms/step")
        return ms

    tiles = tiles or default_tiles(wl.dim, wl.n)
    first = [Choice(t, 4096, k) for t, k in itertools.product(tiles, intervals)]
    best = min(first, key=measure)
    for P in block_sizes:
        if P != best.block_particles:
            ch = Choice(best.tile, P, best.sort_interval)
            if measure(ch) < min(ms for c, ms in table if c == best):
                best = ch
    if cache:
        data = {}
        if os.path.exists(cache):
            try:
                data = json.load(open(cache))
            except ValueError:
                data = {}
        data[key] = {"choice": asdict(best),
                     "table": [[asdict(c), ms] for c, ms in table]}
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return best, table
