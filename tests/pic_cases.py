"""Shared set-up for the GPU parity tests: the same seeded initial state is
given to the CUDA path (through the C ABI) and to the FP64 oracle; each side
converts it to its own representation."""
from __future__ import annotations

import math
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


def field_bound(jtol, steps):
    """Bound on the relative L2 error of E and B after `steps` steps of the
    FP32 path, from the bound jtol on one step's current.  Each half step
    adds (dt/2) J to E, and B follows from the curl of E; the current's
    error comes from rounding each step's moves to integers, which is
    independent from step to step, so the accumulated field error grows like
    a random walk of per-step errors of size jtol: jtol (1 + sqrt(steps)).
    (Measured on the B300 with the thermal parity cases over 20 steps: E
    stays within 1.7 jtol-sized current errors, B grows like steps^0.35-0.5
    and reaches 3.7 times the current's error, under this bound.)"""
    return jtol * (1.0 + math.sqrt(steps))


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


def sampled_push_check(G, wl, sp, t, n_sample=2000, seed=5):
    """One step of species `sp` at full size against the oracle: at the
    start of a step (time t) the grid's first Maxwell half step is taken and
    the species sorted; n_sample particles drawn at random are then pushed
    by the FP64 oracle in the GPU's own fields and by the GPU (all
    particles).  Returns the relative L2 error of the sample's momenta, the
    largest position error in cells (integer-time positions, periodic dimensions
    unwrapped) and the number of nodes where the integer continuity residual
    rho1 - rho0 + div J_int is not zero (interior columns with absorbing x)."""
    import torch
    G.maxwell_half(0, t)
    G.zero_current()
    G.sort(sp.id)
    st = sp.state()
    rng = np.random.Generator(np.random.Philox(seed))
    pick = rng.choice(st["id"].shape[0], size=n_sample, replace=False)
    ids = st["id"][pick]
    rho0 = sp.charge()
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
    G.gather_push_deposit(sp.id)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    st1 = sp.state()
    x1 = sp.positions_at_step()
    order = np.argsort(st1["id"])
    rows = order[np.searchsorted(st1["id"][order], ids)]
    assert np.array_equal(st1["id"][rows], ids)
    alive = osp.alive.astype(bool)
    ug = st1["u"][:, rows[alive]].astype(np.float64)
    uo = osp.u[:, alive]
    rel_u = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
    diff = x1[:, rows[alive]] - osp.x[:wl.dim, alive]
    for d in range(wl.dim):
        if d > 0 or not wl.absorb_x:
            L = wl.n[d] * wl.h[d]
            diff[d] = np.remainder(diff[d] + 0.5 * L, L) - 0.5 * L
    dx = np.max(np.abs(diff) / h)
    rho1 = sp.charge()
    J = G.J
    div = (J[0] - torch.roll(J[0], 1, 2)) + (J[1] - torch.roll(J[1], 1, 1))
    if wl.dim == 3:
        div = div + (J[2] - torch.roll(J[2], 1, 0))
    res = rho1 - rho0 + div
    if wl.absorb_x:
        res = res[:, :, 4:-4]
    return float(rel_u), float(dx), int(torch.count_nonzero(res).item())
