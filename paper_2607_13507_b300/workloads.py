"""Seeded synthetic inputs for the PIC hot path.

This module only draws initial conditions (particle cells, in-cell offsets,
momenta, weights, ids) and describes the workloads.  It holds none of the
method's arithmetic (no push, gather, deposit or field update) and is the one
piece shared by the CUDA path and the CPU oracle used by the tests.

Every random number comes from numpy's Philox4x32-10 counter-based generator
(Salmon et al., SC'11) keyed by an explicit seed.  Offsets, momenta and
weights are rounded to float32-representable values, so the FP32 path, the
FP64 path and the oracle all start from bit-identical states.

Units are normalised (c = eps0 = 1, |e| = m_e = 1).  The thermal workloads use
c/omega_p and 1/omega_p with n0 = 1; the laser workloads use c/omega_0 and
1/omega_0 (lambda = 2 pi) with the critical density n_c = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20261202


def generator(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _f32_unit(a: np.ndarray) -> np.ndarray:
    """float32 values inside [0, 1)."""
    a = a.astype(np.float32, copy=False)
    np.minimum(a, np.nextafter(np.float32(1.0), np.float32(0.0)), out=a)
    np.maximum(a, np.float32(0.0), out=a)
    return a


@dataclass
class Particles:
    """Initial state of one species.

    cell: (dim, n) int32 cell coordinates; off: (dim, n) float32 in-cell
    offsets in [0, 1) (cell units); u: (3, n) float32 momenta u = gamma v;
    w: (n,) float32 weights; id: (n,) int32 particle ids (0..n-1).
    """
    q: float
    m: float
    cell: np.ndarray
    off: np.ndarray
    u: np.ndarray
    w: np.ndarray
    id: np.ndarray

    @property
    def n(self) -> int:
        return int(self.w.shape[0])


@dataclass
class SpeciesSpec:
    q: float
    m: float
    ppc: int
    vth: float                      # per-component momentum spread (u ~ N(0, vth^2))
    # or, with theta > 0, momenta from the Maxwell-Juttner distribution at
    # temperature kT = theta m c^2 (vth unused)
    theta: float = 0.0
    density: float = 1.0            # peak density
    profile: str = "uniform"        # "uniform" | "slab"
    slab: tuple = ()                # (ramp_start, ramp_end, plateau_end) in x, physical units
    same_positions_as: int = -1     # load at the positions of an earlier species


@dataclass
class LaserSpec:
    a0: float
    w0: float
    tau: float                      # full sin^2 envelope duration
    omega: float = 1.0


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    h: tuple
    dt: float
    order: int                      # 1 = CIC, 2 = TSC
    absorb_x: bool
    species: list
    steps: int
    laser: LaserSpec | None = None
    precision: str = "fp32"         # "fp64" | "fp32"
    seed: int = SEED_BASE
    notes: str = ""
    boundary: str = "mur"           # absorbing x: "mur" edges or "cpml" layers
    b0: float = 0.0                 # uniform initial B_z (normalised units)
    qed_eps_ref: float = 0.0        # > 0: nonlinear Compton emission, hbar omega / (m c^2)

    @property
    def cells(self) -> int:
        return int(np.prod(self.n))

    @property
    def dV(self) -> float:
        return float(np.prod(self.h))

    def laser_center(self):
        return tuple(0.5 * self.n[d] * self.h[d] for d in range(1, self.dim))


def cfl_dt(h, eta=0.95) -> float:
    """dt = eta / (c sqrt(sum h^-2)) (Sec. 3.2)."""
    return eta / math.sqrt(sum(1.0 / x ** 2 for x in h))


def _density(spec: SpeciesSpec, xc: np.ndarray) -> np.ndarray:
    if spec.profile == "uniform":
        return np.full(xc.shape, spec.density)
    r0, r1, p1 = spec.slab
    n = np.zeros(xc.shape)
    ramp = (xc >= r0) & (xc < r1)
    n[ramp] = spec.density * (xc[ramp] - r0) / (r1 - r0)
    n[(xc >= r1) & (xc < p1)] = spec.density
    return n


def maxwell_juttner(g: np.random.Generator, theta: float, n: int) -> np.ndarray:
    """Momenta u = gamma v / c (shape (3, n), float64) of n particles drawn
    from the Maxwell-Juttner distribution at temperature kT = theta m c^2:
    isotropic, |u| with density proportional to u^2 exp(-(gamma - 1) / theta).

    Exact rejection sampling on the kinetic energy e = gamma - 1, whose density
    is proportional to sqrt(e (e + 2)) (1 + e) exp(-e / theta).  Because
    sqrt(e + 2) <= sqrt(2) sqrt(1 + e) and (1 + e)^(3/2) <= (1 + e)^2
    <= 2 (1 + e^2), that density lies under 2 sqrt(2) (e^(1/2) + e^(5/2))
    exp(-e / theta), a mixture of two gamma distributions (shapes 3/2 and 7/2,
    scale theta) that numpy samples directly; a candidate is kept with
    probability sqrt(e + 2) (1 + e) / (2 sqrt(2) (1 + e^2)) (at least about
    one half at small theta).  That acceptance falls like 1 / sqrt(e) at large
    energies, so for theta >= 1 the envelope is (1 + e)^2 exp(-e / theta)
    instead (sqrt(e (e + 2)) <= 1 + e): a mixture of gamma distributions of
    shapes 1, 2, 3 with weights theta, 2 theta^2, 2 theta^3, and acceptance
    sqrt(e (e + 2)) / (1 + e), close to one where e >> 1.  Directions are
    uniform on the sphere."""
    out = np.empty(0)
    if theta >= 1.0:
        wts = np.array([theta, 2.0 * theta ** 2, 2.0 * theta ** 3])
        cum = np.cumsum(wts / wts.sum())
        while out.shape[0] < n:
            m = (n - out.shape[0]) * 5 // 4 + 64
            shape = 1.0 + np.searchsorted(cum, g.random(m), side="right").clip(0, 2)
            e = theta * g.standard_gamma(shape)
            keep = g.random(m) * (1.0 + e) <= np.sqrt(e * (e + 2.0))
            out = np.concatenate([out, e[keep]])
    wa = math.gamma(1.5) * theta ** 1.5
    wb = math.gamma(3.5) * theta ** 3.5
    pa = wa / (wa + wb)
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 64
        shape = np.where(g.random(m) < pa, 1.5, 3.5)
        e = theta * g.standard_gamma(shape)
        keep = g.random(m) * (2.0 * math.sqrt(2.0) * (1.0 + e * e)) <= np.sqrt(e + 2.0) * (1.0 + e)
        out = np.concatenate([out, e[keep]])
    e = out[:n]
    umag = np.sqrt(e * (e + 2.0))
    cth = 2.0 * g.random(n) - 1.0
    phi = 2.0 * math.pi * g.random(n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([umag * sth * np.cos(phi), umag * sth * np.sin(phi), umag * cth])


def load_species(wl: Workload, sid: int, previous: list | None = None,
                 cells: tuple | None = None) -> Particles:
    """Exactly ``ppc`` particles per loaded cell, uniform in the cell, with
    momenta u_i ~ N(0, vth^2) (or Maxwell-Juttner at theta) and weight
    w = n(x_cell) dV / ppc.  Cells of zero
    density get no particles.  ``cells`` restricts loading to a box of cells
    ((lo, hi) per dimension) for sampled runs."""
    spec = wl.species[sid]
    g = generator(wl.seed + 1000 * sid)
    dim = wl.dim
    axes = []
    for d in range(dim):
        lo, hi = (0, wl.n[d]) if cells is None else cells[d]
        axes.append(np.arange(lo, hi, dtype=np.int64))
    # cell coordinates, x fastest
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    cc = [m.reshape(-1) for m in mesh[::-1]]            # cc[0] = x index, ...
    xc = (cc[0] + 0.5) * wl.h[0]
    dens = _density(spec, xc)
    keep = dens > 0.0
    cc = [c[keep] for c in cc]
    dens = dens[keep]
    ncell = dens.shape[0]
    ppc = spec.ppc
    n = ncell * ppc
    if spec.same_positions_as >= 0 and previous is not None:
        src = previous[spec.same_positions_as]
        assert src.n == n
        cell = src.cell.copy()
        off = src.off.copy()
    else:
        cell = np.empty((dim, n), dtype=np.int32)
        for d in range(dim):
            cell[d] = np.repeat(cc[d].astype(np.int32), ppc)
        off = _f32_unit(g.random((dim, n), dtype=np.float32))
    if spec.theta > 0.0:
        u = maxwell_juttner(g, spec.theta, n).astype(np.float32)
    else:
        u = g.standard_normal((3, n), dtype=np.float32)
        u *= np.float32(spec.vth)
    w = (np.repeat(dens, ppc) * wl.dV / ppc).astype(np.float32)
    ids = np.arange(n, dtype=np.int32)
    return Particles(spec.q, spec.m, cell, off, u, w, ids)


def load_all(wl: Workload, cells: tuple | None = None) -> list:
    out = []
    for s in range(len(wl.species)):
        out.append(load_species(wl, s, out, cells))
    if wl.qed_eps_ref > 0:
        # the emission draws are keyed by particle id: ids unique across species
        base = 0
        for p in out:
            p.id = (p.id + base).astype(np.int32)
            base += p.n
    return out


# --------------------------------------------------------------- workloads
ELECTRON = dict(q=-1.0, m=1.0)
PROTON = dict(q=1.0, m=1836.0)
LAMBDA = 2.0 * math.pi


def thermal2d(n=64, ppc=16, vth=0.01, order=1, steps=200, precision="fp64", seed=None) -> Workload:
    """2D3V periodic thermal plasma, dx = dy = 0.1 c/omega_p, dt = 0.95 CFL, one
    electron species with a fixed (not deposited) ion background."""
    h = (0.1, 0.1)
    return Workload(f"thermal2d_{n}x{n}_ppc{ppc}", 2, (n, n), h, cfl_dt(h), order, False,
                    [SpeciesSpec(**ELECTRON, ppc=ppc, vth=vth)], steps,
                    precision=precision, seed=SEED_BASE + 1000 * 1 if seed is None else seed)


def laser2d(nx=2048, ny=1024, ppc=32, order=2, steps=1600, precision="fp32", seed=None,
            boundary="mur") -> Workload:
    """2D3V laser-plasma: dx = lambda/32, a0 = 10 laser (waist 4 lambda, 8-cycle
    sin^2 envelope) entering at x-min through an absorbing edge; electron +
    proton slab at 10 n_c with a 2 lambda linear ramp; absorbing x, periodic y.
    The slab sits at the same fractions of the box when nx is scaled down."""
    dx = LAMBDA / 32.0
    h = (dx, dx)
    Lx = nx * dx
    r0, r1, p1 = (16.0 / 64.0) * Lx, (18.0 / 64.0) * Lx, (48.0 / 64.0) * Lx
    sp = [SpeciesSpec(**ELECTRON, ppc=ppc, vth=0.01, density=10.0, profile="slab", slab=(r0, r1, p1)),
          SpeciesSpec(**PROTON, ppc=ppc, vth=0.0, density=10.0, profile="slab", slab=(r0, r1, p1),
                      same_positions_as=0)]
    return Workload(f"laser2d_{nx}x{ny}" + ("_cpml" if boundary == "cpml" else ""), 2, (nx, ny), h,
                    cfl_dt(h), order, True, sp, steps,
                    laser=LaserSpec(a0=10.0, w0=4.0 * LAMBDA, tau=8.0 * LAMBDA),
                    precision=precision, seed=SEED_BASE + 1000 * 2 if seed is None else seed,
                    boundary=boundary)


def thermal3d(n=256, ppc=8, vth=0.05, order=2, steps=100, precision="fp32", seed=None) -> Workload:
    """3D3V periodic thermal plasma, dx = 0.1 c/omega_p, dt = 0.95 CFL, electrons
    with a fixed ion background (the roofline run at n = 256, ppc = 8)."""
    h = (0.1, 0.1, 0.1)
    return Workload(f"thermal3d_{n}^3_ppc{ppc}", 3, (n, n, n), h, cfl_dt(h), order, False,
                    [SpeciesSpec(**ELECTRON, ppc=ppc, vth=vth)], steps,
                    precision=precision, seed=SEED_BASE + 1000 * 3 if seed is None else seed)


def laser3d(nx=512, ny=256, nz=256, ppc=16, order=1, steps=500, precision="fp32", seed=None,
            boundary="mur") -> Workload:
    """3D3V laser-target: dx = lambda/32, a0 = 20 laser (waist 2 lambda, 8-cycle
    envelope) on a 30 n_c slab 2 lambda thick at x in [4, 6] lambda (scaled with
    nx), electrons + protons, absorbing x, periodic y and z."""
    dx = LAMBDA / 32.0
    h = (dx, dx, dx)
    Lx = nx * dx
    r0 = (4.0 / 16.0) * Lx
    r1 = r0 + 1e-9
    p1 = (6.0 / 16.0) * Lx
    sp = [SpeciesSpec(**ELECTRON, ppc=ppc, vth=0.01, density=30.0, profile="slab", slab=(r0, r1, p1)),
          SpeciesSpec(**PROTON, ppc=ppc, vth=0.0, density=30.0, profile="slab", slab=(r0, r1, p1),
                      same_positions_as=0)]
    return Workload(f"laser3d_{nx}x{ny}x{nz}" + ("_cpml" if boundary == "cpml" else ""), 3, (nx, ny, nz), h, cfl_dt(h), order, True, sp, steps,
                    laser=LaserSpec(a0=20.0, w0=2.0 * LAMBDA, tau=8.0 * LAMBDA),
                    precision=precision, seed=SEED_BASE + 1000 * 5 if seed is None else seed,
                    boundary=boundary)


M_E_KEV = 510.999  # electron rest energy, keV


def heating2d(res=20, ppc=16, L_lambda=16, precision="fp32", seed=None) -> Workload:
    """The numerical-heating set-up (Sec. 4.1): a uniform 2D electron-ion
    plasma at n_e = 10 n_c and kT = 1 keV for both species (Maxwell-Juttner
    momenta), periodic in both directions, cell-in-cell shapes, dt = 0.95 CFL,
    evolved for 5000 / omega_pe, dx = lambda / res (20 and 40 in the paper),
    ppc particles per cell and species (16 and 64).  The box side (L_lambda
    wavelengths) and the ion mass (protons) are not given in the paper; the
    ions start at the electrons' positions (a neutral start)."""
    dx = LAMBDA / res
    n = int(round(L_lambda * res))
    h = (dx, dx)
    dt = cfl_dt(h)
    omega_pe = math.sqrt(10.0)
    steps = int(math.ceil(5000.0 / omega_pe / dt))
    sp = [SpeciesSpec(**ELECTRON, ppc=ppc, vth=0.0, density=10.0, theta=1.0 / M_E_KEV),
          SpeciesSpec(**PROTON, ppc=ppc, vth=0.0, density=10.0, theta=1.0 / (M_E_KEV * PROTON["m"]),
                      same_positions_as=0)]
    return Workload(f"heating2d_dx{res}_ppc{ppc}_{n}x{n}", 2, (n, n), h, dt, 1, False, sp, steps,
                    precision=precision, seed=SEED_BASE + 1000 * 6 + res + ppc if seed is None else seed)


def qed2d(n=1024, ppc=16, theta=3000.0, b0=4.0, lambda_um=0.8, order=2, precision="fp32",
          seed=None) -> Workload:
    """Synchrotron cooling of a hot pair plasma through nonlinear Compton
    emission (Sec. 3.4): electrons and positrons at kT = theta m c^2
    (Maxwell-Juttner momenta, mean gamma ~ 3 theta) and density 1 n_c each,
    in a uniform B_z = b0 (units m c omega / e), periodic n x n box of
    lambda / 32 cells, dt = 0.95 CFL; eps_ref = hbar omega / (m c^2) of a
    lambda_um laser.  With the defaults chi ~ eps_ref gamma b0 ~ 0.1 and
    about 0.5% of the leptons emit a photon per step.  The paper gives no
    QED benchmark configuration: this set-up is synthetic.  Positron ids
    follow the electrons' (ids are unique across the emitting species)."""
    dx = LAMBDA / 32
    h = (dx, dx)
    dt = cfl_dt(h)
    sp = [SpeciesSpec(**ELECTRON, ppc=ppc, vth=0.0, density=1.0, theta=theta),
          SpeciesSpec(q=1.0, m=1.0, ppc=ppc, vth=0.0, density=1.0, theta=theta, same_positions_as=0)]
    eps = 1.23984198 / lambda_um / (M_E_KEV * 1e3)
    return Workload(f"qed2d_{n}x{n}_ppc{ppc}", 2, (n, n), h, dt, order, False, sp, 100,
                    precision=precision, b0=b0, qed_eps_ref=eps,
                    seed=SEED_BASE + 1000 * 7 + n + ppc if seed is None else seed)


@dataclass
class EnsembleMember:
    n: tuple
    ppc: int
    vth: float


def ensemble(count=96, lo=128, hi=768, seed=None) -> list:
    """Batched ensemble: independent 2D3V periodic plasmas with sides drawn
    uniformly from [lo, hi], 4..64 particles per cell and v_th in [0.005, 0.1]."""
    g = generator(SEED_BASE + 1000 * 4 if seed is None else seed)
    out = []
    for i in range(count):
        nx, ny = (int(v) for v in g.integers(lo, hi + 1, size=2))
        ppc = int(g.integers(4, 65))
        vth = float(g.uniform(0.005, 0.1))
        out.append(thermal2d(n=nx, ppc=ppc, vth=vth, order=1, steps=100, precision="fp32",
                             seed=SEED_BASE + 1000 * 4 + 1 + i))
        out[-1].n = (nx, ny)
        out[-1].name = f"ens{i}_{nx}x{ny}_ppc{ppc}"
    return out
