"""Shared set-up for the GPU parity tests: the same seeded initial state is
given to the CUDA path (through the C ABI) and to the FP64 oracle; each side
converts it to its own representation."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2607_13507_b300 import workloads as W


def oracle_case(wl: W.Workload, parts):
    laser = None
    if wl.laser is not None:
        c = wl.laser_center()
        laser = O.Laser(wl.laser.a0, wl.laser.w0, wl.laser.tau, wl.laser.omega, c[0],
                        c[1] if wl.dim == 3 else 0.0)
    pml = O.Pml() if getattr(wl, "boundary", "mur") == "cpml" else None
    g = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=wl.absorb_x, laser=laser, pml=pml)
    h = np.array(wl.h)[:, None]
    sps = [O.Species(p.q, p.m, (p.cell + p.off) * h, p.u, p.w) for p in parts]
    return g, sps


def run_oracle(g, sps, steps, t0=0.0):
    for s in range(steps):
        O.step(g, sps, t0 + s * g.dt)


def gpu_case(wl, parts, precision, tile=None):
    from paper_2607_13507_b300 import lpic
    G = lpic.grid_for(wl, precision, tile)
    for p in parts:
        G.add_species(p)
    return G


def run_gpu(G, steps, t0=0.0):
    import torch
    for s in range(steps):
        G.step(t0 + s * G.dt)
    torch.cuda.synchronize()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def match_particles(G, sp_gpu, sp_orc, wl):
    """Alive particles of both sides matched by id: returns (x_gpu, x_orc,
    u_gpu, u_orc) with x the integer-time positions, periodic dimensions
    unwrapped to the representative closest to the oracle's."""
    st = sp_gpu.state()
    x_g = sp_gpu.positions_at_step()
    ids = st["id"]
    alive_o = sp_orc.alive.astype(bool)
    idx_o = np.nonzero(alive_o)[0]
    assert set(ids.tolist()) == set(idx_o.tolist()), "alive sets differ"
    order = np.argsort(ids)
    ids = ids[order]
    xg = x_g[:, order]
    ug = st["u"][:, order].astype(np.float64)
    xo = sp_orc.x[: wl.dim, ids]
    uo = sp_orc.u[:, ids]
    for d in range(wl.dim):
        if d == 0 and wl.absorb_x:
            continue
        L = wl.n[d] * wl.h[d]
        xg[d] = xo[d] + np.remainder(xg[d] - xo[d] + 0.5 * L, L) - 0.5 * L
    return xg, xo, ug, uo
