"""Autotuner for the FP32 path: tile shape, particles per thread block and
sort interval.

Each candidate is timed on the actual workload for a few full steps
(CUDA events on the stepping stream, after warm-up); the fastest wins.  With
pre_steps > 0 the workload is first advanced that many steps (for a laser,
until the pulse is on the target) and every candidate starts from that
snapshot of particles and fields, so the choice fits the state the benchmark
times.  The search is staged to keep it short: tile shape x sort interval at
the default block size, then the other block sizes for the three best pairs.  Results can
be cached in a JSON file keyed by the workload's signature (grid, cell sizes,
shape order, species, particles per cell, boundaries).

Ensembles (`tune_ensemble`): members are grouped by particles per cell, the
quantity that decides how full a tile of a given shape is; one representative
periodic plasma per group is timed alone over the tile shapes and block sizes
(sort every step, as ensembles do), and each member takes its group's best.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from dataclasses import asdict, dataclass

import numpy as np
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


def snapshot(wl, parts, pre_steps, stream, device="cuda"):
    """Advances the workload pre_steps steps (default launch choice) and
    returns its particles (leapfrog-staggered state) and fields."""
    G = lpic.grid_for(wl, lpic.FP32_FIXED, device=device)
    try:
        for p in parts:
            G.add_species(p, stream=stream)
        for s in range(pre_steps):
            G.step(s * G.dt, stream)
        stream.synchronize()
        n = wl.n
        out = []
        for sp, p in zip(G.species, parts):
            st = sp.state(stream)
            c = st["cell"].astype(np.int64)
            coords = [c % n[0], (c // n[0]) % n[1]] + ([c // (n[0] * n[1])] if wl.dim == 3 else [])
            out.append(W.Particles(p.q, p.m, np.stack(coords).astype(np.int32), st["off"], st["u"],
                                   st["w"], st["id"]))
        fields = {"E": [t.clone() for t in G.E], "B": [t.clone() for t in G.B],
                  "J": [t.clone() for t in G.J], "F": G.info().fixed_shift, "step": pre_steps}
        return out, fields
    finally:
        G.close()
        del G
        torch.cuda.empty_cache()


def time_choice(wl, parts, ch: Choice, steps=6, warmup=2, stream=None, device="cuda", fields=None) -> float:
    """Milliseconds per full step of the workload with this choice (from a
    snapshot when `fields` is given)."""
    st = stream or torch.cuda.current_stream()
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=ch.tile, device=device,
                      block_particles=ch.block_particles, sort_interval=ch.sort_interval)
    try:
        s0 = 0
        for p in parts:
            G.add_species(p, staggered=fields is not None, stream=st)
        if fields is not None:
            s0 = fields["step"]
            for name in ("E", "B"):
                for dst, src in zip(getattr(G, name), fields[name]):
                    dst.copy_(src)
            if G.info().fixed_shift == fields["F"]:
                for dst, src in zip(G.J, fields["J"]):
                    dst.copy_(src)
        for s in range(s0, s0 + warmup):
            G.step(s * G.dt, st)
        # a whole number of sort intervals, so every choice pays its sorts
        k = max(1, ch.sort_interval)
        steps = k * ((steps + k - 1) // k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.synchronize()
        a.record(st)
        for s in range(s0 + warmup, s0 + warmup + steps):
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


def autotune(wl: W.Workload, tiles=None, intervals=(1, 2, 4, 8), block_sizes=(2048, 4096, 8192),
             steps=6, warmup=2, cache: str | None = None, log=None, pre_steps=0,
             refresh=False) -> tuple:
    """Returns (best Choice, list of (Choice, ms per step)); a cached result
    is used unless refresh is set."""
    key = signature(wl)
    if cache and not refresh and os.path.exists(cache):
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
    fields = None
    if pre_steps > 0:
        parts, fields = snapshot(wl, parts, pre_steps, stream)

    def measure(ch):
        ms = time_choice(wl, parts, ch, steps, warmup, stream, fields=fields)
        table.append((ch, ms))
        if log:
            log(f"autotune {ch} -> {ms:.3f} ms/step")
        return ms

    tiles = tiles or default_tiles(wl.dim, wl.n)
    first = [Choice(t, 4096, k) for t, k in itertools.product(tiles, intervals)]
    for ch in first:
        measure(ch)
    # the other block sizes for the three best (tile, interval) pairs
    for c0, _ in sorted(table, key=lambda e: e[1])[:3]:
        for P in block_sizes:
            if P != c0.block_particles:
                measure(Choice(c0.tile, P, c0.sort_interval))
    best = min(table, key=lambda e: e[1])[0]
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


def ppc_class(ppc: int) -> int:
    """The power of two nearest to ppc in log scale (members are grouped by it)."""
    return 1 << max(0, int(round(math.log2(max(ppc, 1)))))


def _cache_load(cache):
    if cache and os.path.exists(cache):
        try:
            return json.load(open(cache))
        except ValueError:
            return {}
    return {}


def tune_ensemble(members, tiles=None, block_sizes=(4096, 8192), side=512, vth=0.05, steps=6, warmup=2,
                  cache: str | None = None, log=None, refresh=False) -> tuple:
    """Per-member launch choices for an ensemble of periodic 2D plasmas.
    Returns (one Choice per member, {ppc class: (Choice, table)})."""
    wl0 = members[0]
    classes = sorted({ppc_class(m.species[0].ppc) for m in members})
    data = _cache_load(cache)
    best = {}
    for c in classes:
        key = f"ensemble-class|{wl0.dim}|{wl0.order}|ppc{c}|side{side}"
        rec = None if refresh else data.get(key)
        if rec:
            ch = rec["choice"]
            best[c] = (Choice(tuple(ch["tile"]), ch["block_particles"], 1), rec["table"])
            continue
        rep = W.thermal2d(n=side, ppc=c, vth=vth, order=wl0.order, precision="fp32", seed=W.SEED_BASE + 7000 + c)
        parts = W.load_all(rep)
        stream = torch.cuda.Stream()
        table = []
        for t in (tiles or default_tiles(rep.dim, rep.n)):
            for P in block_sizes:
                ch = Choice(t, P, 1)
                ms = time_choice(rep, parts, ch, steps, warmup, stream)
                table.append((ch, ms))
                if log:
                    log(f"ensemble class ppc {c}: {ch} -> {ms:.3f} ms/step")
        b = min(table, key=lambda e: e[1])[0]
        best[c] = (b, [[asdict(ch), ms] for ch, ms in table])
        data[key] = {"choice": asdict(b), "table": best[c][1],
                     "representative": f"{side}x{side} periodic plasma, {c} particles per cell, v_th {vth}c"}
        if cache:
            with open(cache, "w") as f:
                json.dump(data, f, indent=1)
    choices = [best[ppc_class(m.species[0].ppc)][0] for m in members]
    return choices, best
