"""ctypes wrapper around the FP64 CPU oracle (``lpic_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library.

The oracle computes the explicit electromagnetic PIC timestep of the
lambdaPIC paper (Algorithm 1 without QED / load balancing / MPI): Yee
half-steps (Sec. 3.2, Eq. 1-4), half position pushes, staggered-node gather
and relativistic Boris (Sec. 3.1), Esirkepov deposit (Sec. 3.1).  Positions
are physical coordinates in double precision; fields are ``[nz][ny][fx]``
arrays (``fx = nx`` periodic, ``nx + 1`` with absorbing x edges).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpic_oracle.c")
_SO = os.path.join(_HERE, "_build", "liblpic_oracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no fast-math, no vector ISA flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-D_DEFAULT_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _CGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("fx", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("order", ctypes.c_int), ("absorb_x", ctypes.c_int),
                ("laser", ctypes.c_int), ("a0", ctypes.c_double), ("w0", ctypes.c_double),
                ("tau", ctypes.c_double), ("omega", ctypes.c_double), ("yc", ctypes.c_double),
                ("zc", ctypes.c_double),
                ("E", _dp * 3), ("B", _dp * 3), ("J", _dp * 3),
                ("cpml", ctypes.c_int), ("pml_cells", ctypes.c_int), ("laser_plane", ctypes.c_int),
                ("pml_m", ctypes.c_double), ("pml_sigma_max", ctypes.c_double),
                ("pml_kappa_max", ctypes.c_double), ("pml_alpha_max", ctypes.c_double),
                ("psi", _dp * 4)]


class Pml:
    """CPML layers on the x ends (absorbing x only): cells per layer, grading
    exponent m, sigma_max (None: 0.8 (m + 1) / dx, the usual optimum for
    c = eps0 = 1), kappa_max, alpha_max.  The laser (if any) is a current sheet
    on node plane cells + 2."""

    def __init__(self, cells=16, m=3.0, sigma_max=None, kappa_max=1.0, alpha_max=0.05):
        self.cells, self.m, self.sigma_max = int(cells), float(m), sigma_max
        self.kappa_max, self.alpha_max = float(kappa_max), float(alpha_max)


class _CSpecies(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("n", ctypes.c_long),
                ("x", _dp * 3), ("u", _dp * 3), ("w", _dp), ("alive", _ip)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        _lib.orc_shape.restype = ctypes.c_double
        _lib.orc_shape.argtypes = [ctypes.c_int, ctypes.c_double]
        _lib.orc_laser_ey.restype = ctypes.c_double
        _lib.orc_laser_ey.argtypes = [ctypes.POINTER(_CGrid)] + [ctypes.c_double] * 4
        _lib.orc_gather.argtypes = [ctypes.POINTER(_CGrid), _dp, _dp, _dp]
        _lib.orc_boris.argtypes = [ctypes.c_double] * 3 + [_dp, _dp, _dp]
        _lib.orc_boris.restype = None
        _lib.orc_deposit.argtypes = [ctypes.POINTER(_CGrid), ctypes.c_double, _dp, _dp,
                                     ctypes.c_double]
        _lib.orc_rho.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies), _dp]
        _lib.orc_maxwell_half.argtypes = [ctypes.POINTER(_CGrid), ctypes.c_int, ctypes.c_double]
        _lib.orc_maxwell_half.restype = None
        _lib.orc_push_species.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies)]
        _lib.orc_step.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies),
                                  ctypes.c_int, ctypes.c_double]
        _lib.orc_energy.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies),
                                    ctypes.c_int, _dp]
        _lib.orc_energy.restype = None
        _lib.orc_div_e.argtypes = [ctypes.POINTER(_CGrid), _dp]
        _lib.orc_div_e.restype = None
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Laser:
    """Incoming E_y-polarised laser at x-min (Sec. 4.2: Gaussian spot, sin^2
    envelope); ``tau`` is the full envelope duration."""

    def __init__(self, a0, w0, tau, omega=1.0, yc=0.0, zc=0.0):
        self.a0, self.w0, self.tau, self.omega, self.yc, self.zc = a0, w0, tau, omega, yc, zc


class Grid:
    """Yee grid: E, B, J as float64 arrays of shape (nz, ny, fx)."""

    def __init__(self, dim, n, h, dt, order, absorb_x=False, laser: Laser | None = None,
                 pml: Pml | None = None):
        nx, ny = int(n[0]), int(n[1])
        nz = int(n[2]) if dim == 3 else 1
        self.dim, self.nx, self.ny, self.nz = dim, nx, ny, nz
        self.fx = nx + 1 if absorb_x else nx
        self.dx, self.dy = float(h[0]), float(h[1])
        self.dz = float(h[2]) if dim == 3 else 1.0
        self.dt, self.order, self.absorb_x = float(dt), int(order), bool(absorb_x)
        shape = (nz, ny, self.fx)
        self.E = [np.zeros(shape) for _ in range(3)]
        self.B = [np.zeros(shape) for _ in range(3)]
        self.J = [np.zeros(shape) for _ in range(3)]
        self.laser = laser
        assert pml is None or absorb_x, "CPML layers need absorbing x"
        self.pml = pml
        self.psi = [np.zeros(shape) for _ in range(4)]

    @property
    def dV(self):
        return self.dx * self.dy * (self.dz if self.dim == 3 else 1.0)

    def c(self) -> _CGrid:
        L = self.laser
        g = _CGrid(self.dim, self.nx, self.ny, self.nz, self.fx, self.dx, self.dy, self.dz,
                   self.dt, self.order, int(self.absorb_x), int(L is not None),
                   L.a0 if L else 0.0, L.w0 if L else 1.0, L.tau if L else 0.0,
                   L.omega if L else 1.0, L.yc if L else 0.0, L.zc if L else 0.0)
        for c in range(3):
            for name in ("E", "B", "J"):
                arr = getattr(self, name)[c]
                assert arr.dtype == np.float64 and arr.flags.c_contiguous
                getattr(g, name)[c] = _ptr(arr)
        P = self.pml
        if P is not None:
            g.cpml, g.pml_cells, g.laser_plane = 1, P.cells, P.cells + 2
            g.pml_m = P.m
            g.pml_sigma_max = 0.8 * (P.m + 1.0) / self.dx if P.sigma_max is None else float(P.sigma_max)
            g.pml_kappa_max, g.pml_alpha_max = P.kappa_max, P.alpha_max
        for c in range(4):
            g.psi[c] = _ptr(self.psi[c])
        return g


class Species:
    """Particles of one species: x (3, n) physical positions, u (3, n), w (n,), alive (n,)."""

    def __init__(self, q, m, x, u, w, alive=None):
        self.q, self.m = float(q), float(m)
        x = np.asarray(x, dtype=np.float64)
        self.n = x.shape[1]
        self.x = np.zeros((3, self.n))
        self.x[: x.shape[0]] = x
        self.u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3, self.n))
        self.w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(self.n))
        self.alive = (np.ones(self.n, dtype=np.int32) if alive is None
                      else np.ascontiguousarray(np.asarray(alive, dtype=np.int32)))

    def c(self) -> _CSpecies:
        s = _CSpecies(self.q, self.m, self.n)
        for d in range(3):
            s.x[d] = _ptr(self.x[d])
            s.u[d] = _ptr(self.u[d])
        s.w = _ptr(self.w)
        s.alive = self.alive.ctypes.data_as(_ip)
        return s


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} returned {rc}")


def shape(order: int, d: float) -> float:
    return lib().orc_shape(order, d)


def laser_ey(grid: Grid, x, y, z, t) -> float:
    g = grid.c()
    return lib().orc_laser_ey(ctypes.byref(g), x, y, z, t)


def gather(grid: Grid, pos):
    p = np.zeros(3)
    p[: len(pos)] = pos
    E, B = np.zeros(3), np.zeros(3)
    g = grid.c()
    _check(lib().orc_gather(ctypes.byref(g), _ptr(p), _ptr(E), _ptr(B)), "gather")
    return E, B


def boris(q, m, dt, u, E, B):
    u = np.array(u, dtype=np.float64)
    lib().orc_boris(q, m, dt, _ptr(u), _ptr(np.asarray(E, np.float64).copy()),
                    _ptr(np.asarray(B, np.float64).copy()))
    return u


def deposit(grid: Grid, qw, x0, x1, vz=0.0):
    a, b = np.zeros(3), np.zeros(3)
    a[: len(x0)] = x0
    b[: len(x1)] = x1
    g = grid.c()
    _check(lib().orc_deposit(ctypes.byref(g), qw, _ptr(a), _ptr(b), vz), "deposit")


def rho(grid: Grid, sp: Species) -> np.ndarray:
    out = np.zeros((grid.nz, grid.ny, grid.fx))
    g, s = grid.c(), sp.c()
    _check(lib().orc_rho(ctypes.byref(g), ctypes.byref(s), _ptr(out)), "rho")
    return out


def div_e(grid: Grid) -> np.ndarray:
    out = np.zeros((grid.nz, grid.ny, grid.fx))
    g = grid.c()
    lib().orc_div_e(ctypes.byref(g), _ptr(out))
    return out


def maxwell_half(grid: Grid, which: int, t: float = 0.0):
    g = grid.c()
    lib().orc_maxwell_half(ctypes.byref(g), which, t)


def push_species(grid: Grid, sp: Species):
    g, s = grid.c(), sp.c()
    _check(lib().orc_push_species(ctypes.byref(g), ctypes.byref(s)), "push")


def step(grid: Grid, species: list[Species], t: float = 0.0):
    g = grid.c()
    arr = (_CSpecies * len(species))(*[s.c() for s in species])
    _check(lib().orc_step(ctypes.byref(g), arr, len(species), t), "step")


def energy(grid: Grid, species: list[Species]):
    """(kinetic, field, total charge)."""
    g = grid.c()
    arr = (_CSpecies * max(1, len(species)))(*[s.c() for s in species])
    out = np.zeros(3)
    lib().orc_energy(ctypes.byref(g), arr, len(species), _ptr(out))
    return out


# ------------------------------------------------------------------ QED (Sec. 3.4)
def philox(ctr, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key (4 uint32)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(v) for v in o]


def _qed_sigs():
    L = lib()
    d = ctypes.c_double
    for name, res, args in (("orc_bessel_k", d, [d, d]), ("orc_bessel_k_int", d, [d, d]),
                            ("orc_compton_s", d, [d, d]), ("orc_compton_rate", d, [d, d, d]),
                            ("orc_compton_xi", d, [d, d]), ("orc_qed_initial_tau", d,
                                                            [ctypes.c_long, ctypes.c_uint32, ctypes.c_uint32])):
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    L.orc_chi_e.restype = d
    L.orc_chi_e.argtypes = [_dp, _dp, _dp, d]
    for name, res, args in (("orc_bw_f", d, [d, d]), ("orc_bw_rate", d, [d, d, d]), ("orc_bw_eta", d, [d, d]),
                            ("orc_qed_initial_tau_kind", d,
                             [ctypes.c_long, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32])):
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    L.orc_chi_g.restype = d
    L.orc_chi_g.argtypes = [_dp, _dp, _dp, d]
    return L


def bessel_k(nu, x):
    return _qed_sigs().orc_bessel_k(nu, x)


def bessel_k_int(nu, x):
    """int_x^inf K_nu(s) ds"""
    return _qed_sigs().orc_bessel_k_int(nu, x)


def compton_s(xi, chi):
    return _qed_sigs().orc_compton_s(xi, chi)


def compton_rate(chi, gamma, eps_ref):
    return _qed_sigs().orc_compton_rate(chi, gamma, eps_ref)


def compton_xi(chi, r):
    return _qed_sigs().orc_compton_xi(chi, r)


def chi_e(u, E, B, eps_ref):
    a = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (u, E, B)]
    return _qed_sigs().orc_chi_e(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), eps_ref)


def qed_initial_tau(ids, seed):
    L = _qed_sigs()
    lo, hi = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    return np.array([L.orc_qed_initial_tau(int(i), lo, hi) for i in ids])


def qed_compton(grid: Grid, sp: Species, eps_ref, seed, step, tau, cap=1 << 16):
    """Events of one step (after the push); returns the emitted photons as a
    Species (q = 0, m = 0) with positions, momenta and weights."""
    L = lib()
    L.orc_qed_compton.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies), ctypes.c_double,
                                  ctypes.c_uint32, ctypes.c_uint32, ctypes.c_long, _dp, _dp,
                                  ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    g, s = grid.c(), sp.c()
    ph = np.zeros(7 * cap)
    nph = ctypes.c_long(0)
    assert tau.dtype == np.float64 and tau.flags.c_contiguous
    _check(L.orc_qed_compton(ctypes.byref(g), ctypes.byref(s), eps_ref, int(seed) & 0xFFFFFFFF,
                             (int(seed) >> 32) & 0xFFFFFFFF, int(step), _ptr(tau), _ptr(ph), cap,
                             ctypes.byref(nph)), "qed")
    n = nph.value
    ph = ph.reshape(7, cap)[:, :n]
    return Species(0.0, 0.0, ph[:grid.dim].copy(), ph[3:6].copy(), ph[6].copy())


def push_species_qed(grid: Grid, sp: Species, eps_ref, seed, step, tau, cap=1 << 16):
    """One push of `sp` with nonlinear Compton emission between the gather and
    the momentum push (Algorithm 1); returns the emitted photons as a Species
    (positions at the end of the step) and the index of each photon's emitter."""
    L = lib()
    L.orc_push_species_qed.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies), ctypes.c_double,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_long, _dp, _dp,
                                       ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    g, s = grid.c(), sp.c()
    ph = np.zeros(8 * cap)
    nph = ctypes.c_long(0)
    assert tau.dtype == np.float64 and tau.flags.c_contiguous
    _check(L.orc_push_species_qed(ctypes.byref(g), ctypes.byref(s), eps_ref, int(seed) & 0xFFFFFFFF,
                                  (int(seed) >> 32) & 0xFFFFFFFF, int(step), _ptr(tau), _ptr(ph), cap,
                                  ctypes.byref(nph)), "push qed")
    n = nph.value
    ph = ph.reshape(8, cap)[:, :n]
    return Species(0.0, 0.0, ph[:grid.dim].copy(), ph[3:6].copy(), ph[6].copy()), ph[7].astype(np.int64)


# Breit-Wheeler pair creation (Sec. 3.4)
def bw_f(eta, chi):
    return _qed_sigs().orc_bw_f(eta, chi)


def bw_rate(chi, k, eps_ref):
    return _qed_sigs().orc_bw_rate(chi, k, eps_ref)


def bw_eta(chi, r):
    return _qed_sigs().orc_bw_eta(chi, r)


def chi_g(k, E, B, eps_ref):
    a = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (k, E, B)]
    return _qed_sigs().orc_chi_g(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), eps_ref)


def qed_initial_tau_kind(ids, kind, seed):
    """-ln r with r from counter (id, 0, kind, 0): kind 2 for leptons, 3 for photons."""
    L = _qed_sigs()
    lo, hi = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    return np.array([L.orc_qed_initial_tau_kind(int(i), int(kind), lo, hi) for i in ids])


def qed_bw(grid: Grid, ph: Species, eps_ref, seed, step, tau, cap=1 << 16):
    """Pair events of one step; removes converted photons from `ph` and
    returns (electrons, positrons) as Species (q = -1 / +1, m = 1)."""
    L = lib()
    L.orc_qed_bw.argtypes = [ctypes.POINTER(_CGrid), ctypes.POINTER(_CSpecies), ctypes.c_double,
                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_long, _dp, _dp, _dp,
                             ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    g, s = grid.c(), ph.c()
    pe, pp = np.zeros(7 * cap), np.zeros(7 * cap)
    npair = ctypes.c_long(0)
    assert tau.dtype == np.float64 and tau.flags.c_contiguous
    _check(L.orc_qed_bw(ctypes.byref(g), ctypes.byref(s), eps_ref, int(seed) & 0xFFFFFFFF,
                        (int(seed) >> 32) & 0xFFFFFFFF, int(step), _ptr(tau), _ptr(pe), _ptr(pp), cap,
                        ctypes.byref(npair)), "qed bw")
    n = npair.value
    out = []
    for arr, q in ((pe, -1.0), (pp, 1.0)):
        a = arr.reshape(7, cap)[:, :n]
        out.append(Species(q, 1.0, a[:grid.dim].copy(), a[3:6].copy(), a[6].copy()))
    return out[0], out[1]
