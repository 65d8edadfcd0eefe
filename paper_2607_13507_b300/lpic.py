"""Thin ctypes binding of liblpic (include/lpic.h).

Argument marshalling only: PyTorch provides device memory and streams, every
step of the PIC path runs in the CUDA kernels of ``csrc/``.  There is no CPU
fallback: importing this module on a machine without the built library, or
using it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# LPIC_LIBRARY selects another build of the same ABI (the checked library
# liblpic_check.so in the bounds tests)
LIB_PATH = os.environ.get("LPIC_LIBRARY") or os.path.join(_PKG, "_lib", "liblpic.so")

FP64, FP32_FIXED = 0, 1
ST_CFL, ST_HALO, ST_NAN, ST_OUTSIDE, ST_OVERFLOW, ST_BOUNDS = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20

STATUS = {0: "LPIC_OK", 1: "LPIC_EINVAL", 2: "LPIC_ENOMEM", 3: "LPIC_ECUDA", 4: "LPIC_EDEVICE",
          5: "LPIC_EUNSUPPORTED"}

EXPORTS = ["lpic_species_bytes", "lpic_create_grid", "lpic_destroy_grid", "lpic_add_species",
           "lpic_species_query", "lpic_sort_particles", "lpic_zero_current",
           "lpic_gather_push_deposit", "lpic_maxwell_half_step", "lpic_step",
           "lpic_deposit_charge", "lpic_div_e", "lpic_positions_at_step", "lpic_diagnostics",
           "lpic_gather_fields", "lpic_push_deposit_fields", "lpic_step_resolved",
           "lpic_grid_get_info", "lpic_check_status", "lpic_last_error", "lpic_set_clock",
           "lpic_graph_steps", "lpic_sort_tiles_static", "lpic_kernel_timing",
           "lpic_kernel_time", "lpic_create_ensemble", "lpic_destroy_ensemble",
           "lpic_ensemble_step", "lpic_ensemble_graph_steps", "lpic_ensemble_check_status",
           "lpic_ensemble_launches", "lpic_qed_init", "lpic_qed_initial_tau", "lpic_qed_compton",
           "lpic_qed_eval", "lpic_qed_breit_wheeler", "lpic_qed_pair_eval", "lpic_species_set_next_id",
           "lpic_qed_fuse", "lpic_qed_set_step", "lpic_debug_fail_alloc", "lpic_species_checkpoint_info"]


class LpicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class LaserDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("a0", "w0", "tau", "omega", "yc", "zc")]


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("absorb_x", ctypes.c_int),
                ("shape_order", ctypes.c_int), ("precision", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("block_particles", ctypes.c_int),
                ("sort_interval", ctypes.c_int),
                ("E", ctypes.c_void_p * 3), ("B", ctypes.c_void_p * 3),
                ("J", ctypes.c_void_p * 3), ("laser", ctypes.POINTER(LaserDesc)),
                ("pml_cells", ctypes.c_int), ("pml_m", ctypes.c_double),
                ("pml_sigma_max", ctypes.c_double), ("pml_kappa_max", ctypes.c_double),
                ("pml_alpha_max", ctypes.c_double), ("maxwell_fp64", ctypes.c_int)]


class PmlSpec:
    """CPML layers for absorbing x: cells per layer, grading exponent m,
    sigma_max (None: 0.8 (m + 1) / dx), kappa_max, alpha_max."""

    def __init__(self, cells=16, m=3.0, sigma_max=None, kappa_max=1.0, alpha_max=0.05):
        self.cells, self.m, self.sigma_max = int(cells), float(m), sigma_max
        self.kappa_max, self.alpha_max = float(kappa_max), float(alpha_max)


class SpeciesDesc(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("count", ctypes.c_longlong),
                ("capacity", ctypes.c_longlong), ("buffers", ctypes.c_void_p * 2),
                ("staggered", ctypes.c_int), ("max_weight", ctypes.c_double)]


class GridInfo(ctypes.Structure):
    _fields_ = [("fixed_shift", ctypes.c_int), ("j_scale", ctypes.c_double * 3),
                ("rho_scale", ctypes.c_double), ("tile", ctypes.c_int * 3),
                ("ntiles", ctypes.c_longlong), ("fx", ctypes.c_int), ("launches", ctypes.c_longlong)]


class Diag(ctypes.Structure):
    _fields_ = [("kinetic", ctypes.c_double), ("field", ctypes.c_double),
                ("charge", ctypes.c_double), ("particles", ctypes.c_longlong)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblpic.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblpic not built at {path}; run `python -m paper_2607_13507_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    lib.lpic_species_bytes.restype = ctypes.c_size_t
    lib.lpic_species_bytes.argtypes = [i, i, ctypes.c_longlong]
    lib.lpic_create_grid.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)]
    lib.lpic_destroy_grid.argtypes = [vp]
    lib.lpic_add_species.argtypes = [vp, ctypes.POINTER(SpeciesDesc), st, ctypes.POINTER(i)]
    lib.lpic_species_query.argtypes = [vp, i, st, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
    lib.lpic_sort_particles.argtypes = [vp, i, st]
    lib.lpic_zero_current.argtypes = [vp, st]
    lib.lpic_gather_push_deposit.argtypes = [vp, i, st]
    lib.lpic_maxwell_half_step.argtypes = [vp, i, ctypes.c_double, st]
    lib.lpic_step.argtypes = [vp, ctypes.c_double, st]
    lib.lpic_set_clock.argtypes = [vp, ctypes.c_double, st]
    lib.lpic_graph_steps.argtypes = [vp, i, st]
    lib.lpic_kernel_timing.argtypes = [vp, i]
    lib.lpic_create_ensemble.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
    lib.lpic_destroy_ensemble.argtypes = [vp]
    lib.lpic_ensemble_step.argtypes = [vp, st]
    lib.lpic_ensemble_graph_steps.argtypes = [vp, i, st]
    lib.lpic_ensemble_check_status.argtypes = [vp, st, ctypes.POINTER(ctypes.c_uint)]
    lib.lpic_ensemble_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.lpic_kernel_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.lpic_sort_tiles_static.argtypes = [i, i, i, i, ctypes.POINTER(i), vp, vp, ctypes.c_longlong,
                                           vp, vp, vp, st]
    lib.lpic_deposit_charge.argtypes = [vp, i, vp, st]
    lib.lpic_div_e.argtypes = [vp, vp, st]
    lib.lpic_gather_fields.argtypes = [vp, i, vp, st]
    lib.lpic_push_deposit_fields.argtypes = [vp, i, vp, st]
    lib.lpic_step_resolved.argtypes = [vp, ctypes.c_double, i, vp, st]
    lib.lpic_positions_at_step.argtypes = [vp, i, vp, st]
    lib.lpic_diagnostics.argtypes = [vp, ctypes.POINTER(Diag), st]
    lib.lpic_grid_get_info.argtypes = [vp, ctypes.POINTER(GridInfo)]
    lib.lpic_check_status.argtypes = [vp, st, ctypes.POINTER(ctypes.c_uint)]
    lib.lpic_qed_init.argtypes = [vp, ctypes.c_double, ctypes.c_uint64, st]
    lib.lpic_qed_initial_tau.argtypes = [vp, vp, ctypes.c_longlong, i, st]
    lib.lpic_qed_compton.argtypes = [vp, i, i, vp, ctypes.c_longlong, vp, ctypes.c_longlong,
                                     ctypes.c_longlong, st]
    lib.lpic_qed_eval.argtypes = [vp, vp, vp, ctypes.c_longlong, vp, vp, st]
    lib.lpic_qed_breit_wheeler.argtypes = [vp, i, i, i, vp, ctypes.c_longlong, ctypes.c_longlong, st]
    lib.lpic_qed_pair_eval.argtypes = [vp, vp, vp, ctypes.c_longlong, vp, vp, st]
    lib.lpic_species_set_next_id.argtypes = [vp, i, ctypes.c_longlong, st]
    lib.lpic_species_checkpoint_info.argtypes = [vp, i, st, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_longlong)]
    lib.lpic_qed_fuse.argtypes = [vp, i, i, vp, ctypes.c_longlong, vp, ctypes.c_longlong, ctypes.c_longlong, st]
    lib.lpic_qed_set_step.argtypes = [vp, ctypes.c_longlong, st]
    lib.lpic_debug_fail_alloc.argtypes = [ctypes.c_longlong]
    lib.lpic_last_error.restype = ctypes.c_char_p
    lib.lpic_last_error.argtypes = []
    for name in EXPORTS:
        fn = getattr(lib, name)
        # without argtypes ctypes would pass device pointers as 32-bit ints
        if fn.argtypes is None:
            raise RuntimeError(f"{name}: no argument types declared in the binding")
        if name != "lpic_species_bytes" and name != "lpic_last_error":
            fn.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise LpicError(rc, load().lpic_last_error().decode())


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def species_bytes(dim, precision, capacity) -> int:
    return int(load().lpic_species_bytes(dim, precision, capacity))


def _cap(n: int) -> int:
    return max(64, (n + 63) // 64 * 64)


class Species:
    """Device buffers of one species (ping/pong, struct of arrays)."""

    def __init__(self, grid: "Grid", q, m, capacity):
        self.grid, self.q, self.m, self.cap = grid, float(q), float(m), int(capacity)
        nbytes = species_bytes(grid.dim, grid.precision, self.cap)
        self.buffers = [torch.empty(nbytes // 8 + 64, dtype=torch.int64, device=grid.device)
                        for _ in range(2)]
        self.id = -1

    def ptr(self, b) -> int:
        p = self.buffers[b].data_ptr()
        return (p + 255) // 256 * 256

    def _views(self, b):
        """Typed views (cell, off, u, w, id) or (x, u, w, id) of buffer b."""
        g, cap = self.grid, self.cap
        raw = self.buffers[b].view(torch.uint8)
        base = self.ptr(b) - self.buffers[b].data_ptr()
        if g.precision == FP32_FIXED:
            a = 4 * cap
            seg = lambda k, dt: raw[base + k * a: base + (k + 1) * a].view(dt)
            return dict(cell=seg(0, torch.int32),
                        off=[seg(1 + d, torch.float32) for d in range(g.dim)],
                        u=[seg(1 + g.dim + c, torch.float32) for c in range(3)],
                        w=seg(4 + g.dim, torch.float32), id=seg(5 + g.dim, torch.int32))
        a = 8 * cap
        seg = lambda k, dt, sz=a: raw[base + k * a: base + k * a + sz].view(dt)
        return dict(x=[seg(d, torch.float64) for d in range(g.dim)],
                    u=[seg(g.dim + c, torch.float64) for c in range(3)],
                    w=seg(g.dim + 3, torch.float64), id=seg(g.dim + 4, torch.int32, 4 * cap))

    def upload(self, p, staggered=False, stream=None, max_weight=0.0):
        """Copy a workloads.Particles initial state into buffer 0 and register
        the species with the grid."""
        g = self.grid
        n = p.n
        assert n <= self.cap
        v = self._views(0)
        dev = g.device
        if g.precision == FP32_FIXED:
            nx, ny = g.n[0], g.n[1]
            cell = p.cell[0] + nx * (p.cell[1] + (ny * p.cell[2] if g.dim == 3 else 0))
            v["cell"].fill_(-1)
            v["cell"][:n] = torch.from_numpy(cell.astype(np.int32)).to(dev)
            for d in range(g.dim):
                v["off"][d][:n] = torch.from_numpy(p.off[d].astype(np.float32)).to(dev)
            for c in range(3):
                v["u"][c][:n] = torch.from_numpy(p.u[c].astype(np.float32)).to(dev)
            v["w"][:n] = torch.from_numpy(p.w.astype(np.float32)).to(dev)
        else:
            for d in range(g.dim):
                v["x"][d][:n] = torch.from_numpy(
                    (p.cell[d].astype(np.float64) + p.off[d].astype(np.float64)) * g.h[d]).to(dev)
            for c in range(3):
                v["u"][c][:n] = torch.from_numpy(p.u[c].astype(np.float64)).to(dev)
            v["w"].zero_()
            v["w"][:n] = torch.from_numpy(p.w.astype(np.float64)).to(dev)
        v["id"][:n] = torch.from_numpy(p.id).to(dev)
        desc = SpeciesDesc(self.q, self.m, n, self.cap, (ctypes.c_void_p * 2)(self.ptr(0), self.ptr(1)),
                           int(staggered), float(max_weight))
        sid = ctypes.c_int(-1)
        _check(load().lpic_add_species(g.h_, ctypes.byref(desc), _stream(stream), ctypes.byref(sid)))
        self.id = sid.value
        return self

    def query(self, stream=None):
        cur, cnt = ctypes.c_int(), ctypes.c_longlong()
        _check(load().lpic_species_query(self.grid.h_, self.id, _stream(stream), ctypes.byref(cur),
                                         ctypes.byref(cnt)))
        return cur.value, cnt.value

    def state(self, stream=None):
        """Host copy of the current buffer's alive particles as numpy arrays."""
        cur, cnt = self.query(stream)
        v = self._views(cur)
        out = {}
        for k, val in v.items():
            if isinstance(val, list):
                out[k] = np.stack([t[:cnt].cpu().numpy() for t in val])
            else:
                out[k] = val[:cnt].cpu().numpy()
        return out

    def positions_at_step(self, stream=None) -> np.ndarray:
        """x^n (physical, not wrapped) of the current buffer's first count entries."""
        cur, cnt = self.query(stream)
        out = torch.empty(3 * self.cap, dtype=torch.float64, device=self.grid.device)
        _check(load().lpic_positions_at_step(self.grid.h_, self.id, out.data_ptr(), _stream(stream)))
        o = out.view(3, self.cap)[: self.grid.dim, :cnt].cpu().numpy()
        return o

    def set_next_id(self, next_id, stream=None):
        """Id of the next particle this species gains on the device (photons, pairs)."""
        _check(load().lpic_species_set_next_id(self.grid.h_, self.id, int(next_id), _stream(stream)))

    def charge(self, stream=None) -> torch.Tensor:
        """Charge density of the stored positions: float64 (FP64 path) or the
        int64 fixed-point integer charge (FP32 path)."""
        g = self.grid
        dt = torch.float64 if g.precision == FP64 else torch.int64
        rho = torch.zeros(g.field_shape, dtype=dt, device=g.device)
        _check(load().lpic_deposit_charge(g.h_, self.id, rho.data_ptr(), _stream(stream)))
        return rho


class Grid:
    """A grid with caller-owned (torch) field arrays and its species."""

    def __init__(self, dim, n, h, dt, order, precision, absorb_x=False, laser=None, tile=None,
                 device="cuda", block_particles=0, sort_interval=0, pml: PmlSpec | None = None,
                 maxwell_fp64=False):
        load()
        self.dim, self.precision, self.order = dim, precision, order
        self.maxwell_fp64 = bool(maxwell_fp64)
        self.n = tuple(int(v) for v in n) + ((1,) if dim == 2 else ())
        self.h = tuple(float(v) for v in h) + ((1.0,) if dim == 2 else ())
        self.dt, self.absorb_x = float(dt), bool(absorb_x)
        self.device = torch.device(device)
        fx = self.n[0] + 1 if absorb_x else self.n[0]
        nz = self.n[2] if dim == 3 else 1
        self.field_shape = (nz, self.n[1], fx)
        ft = torch.float64 if (precision == FP64 or self.maxwell_fp64) else torch.float32
        jt = torch.float64 if precision == FP64 else torch.int64
        self.E = [torch.zeros(self.field_shape, dtype=ft, device=self.device) for _ in range(3)]
        self.B = [torch.zeros(self.field_shape, dtype=ft, device=self.device) for _ in range(3)]
        self.J = [torch.zeros(self.field_shape, dtype=jt, device=self.device) for _ in range(3)]
        t = tile or (0, 0, 0)
        self._laser = None
        if laser is not None:
            self._laser = LaserDesc(laser.a0, laser.w0, laser.tau, laser.omega, laser.yc, laser.zc)
        if pml is not None and not absorb_x:
            raise ValueError("CPML layers need absorbing x")
        mode = 0 if not absorb_x else (2 if pml is not None else 1)
        self.cpml = mode == 2
        P = pml or PmlSpec(cells=0)
        smax = 0.8 * (P.m + 1.0) / self.h[0] if P.sigma_max is None else float(P.sigma_max)
        desc = GridDesc(dim, self.n[0], self.n[1], nz, self.h[0], self.h[1], self.h[2], self.dt,
                        mode, order, precision, (ctypes.c_int * 3)(*t), int(block_particles), int(sort_interval),
                        (ctypes.c_void_p * 3)(*[a.data_ptr() for a in self.E]),
                        (ctypes.c_void_p * 3)(*[a.data_ptr() for a in self.B]),
                        (ctypes.c_void_p * 3)(*[a.data_ptr() for a in self.J]),
                        ctypes.pointer(self._laser) if self._laser is not None else None,
                        P.cells, P.m, smax, P.kappa_max, P.alpha_max, int(self.maxwell_fp64))
        h = ctypes.c_void_p()
        _check(load().lpic_create_grid(ctypes.byref(desc), ctypes.byref(h)))
        self.h_ = h
        self.species: list[Species] = []

    def close(self):
        if getattr(self, "h_", None):
            load().lpic_destroy_grid(self.h_)
            self.h_ = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_species(self, p, capacity=None, staggered=False, stream=None, max_weight=0.0) -> Species:
        sp = Species(self, p.q, p.m, capacity or _cap(p.n))
        sp.upload(p, staggered, stream, max_weight)
        self.species.append(sp)
        return sp

    def add_empty_species(self, q, m, capacity, stream=None, max_weight=0.0) -> Species:
        """A species that starts empty (m = 0, q = 0: photons created by qed_compton)."""
        from .workloads import Particles
        e = np.zeros((self.dim, 0), np.int32)
        p = Particles(q=q, m=m, cell=e, off=e.astype(np.float32), u=np.zeros((3, 0), np.float32),
                      w=np.zeros(0, np.float32), id=np.zeros(0, np.int32))
        sp = Species(self, q, m, _cap(capacity))
        sp.upload(p, True, stream, max_weight)
        self.species.append(sp)
        return sp

    # -- nonlinear Compton emission
    # -- checkpoint / resume: all state is caller-owned tensors plus the
    # species' weight bounds and id counters; a grid created with the same
    # description restores it and continues bit for bit (FP32 path; the FP64
    # path's double atomics add in a varying order)
    def checkpoint(self, stream=None) -> dict:
        """Host copy of the state: fields, current, fixed-point shift and, per
        species, its charge, mass, capacity, weight bound, next created id
        and the alive particles (leapfrog-staggered)."""
        if self.cpml:
            # the layers' convolution memory lives in the library's scratch
            raise ValueError("checkpoints do not cover the CPML layers' memory")
        torch.cuda.synchronize(self.device)
        out = {"dim": self.dim, "precision": self.precision, "n": list(self.n[:self.dim]),
               "E": [t.cpu().numpy() for t in self.E], "B": [t.cpu().numpy() for t in self.B],
               "J": [t.cpu().numpy() for t in self.J], "species": []}
        if self.precision == FP32_FIXED:
            out["fixed_shift"] = self.info().fixed_shift
        for sp in self.species:
            wmax, nid = ctypes.c_double(), ctypes.c_longlong()
            _check(load().lpic_species_checkpoint_info(self.h_, sp.id, _stream(stream), ctypes.byref(wmax),
                                                       ctypes.byref(nid)))
            st = sp.state(stream)
            key = "cell" if self.precision == FP32_FIXED else "x"
            alive = st[key] >= 0 if key == "cell" else np.ones(st["id"].shape[0], bool)
            parts = {k: (v[..., alive] if v.ndim > 1 else v[alive]) for k, v in st.items()}
            out["species"].append({"q": sp.q, "m": sp.m, "cap": sp.cap, "max_weight": wmax.value,
                                   "next_id": nid.value, "particles": parts})
        return out

    def restore(self, ckpt: dict, stream=None):
        """Load a checkpoint into this grid, created with the same description
        and holding no species yet."""
        from .workloads import Particles
        if self.species:
            raise ValueError("restore needs a grid without species")
        if ckpt["dim"] != self.dim or ckpt["precision"] != self.precision or \
                list(ckpt["n"]) != list(self.n[:self.dim]):
            raise ValueError("checkpoint of another grid description")
        nx, ny = self.n[0], self.n[1]
        for rec in ckpt["species"]:
            st = rec["particles"]
            n = st["id"].shape[0]
            if self.precision == FP32_FIXED:
                c = st["cell"].astype(np.int64)
                coords = [c % nx, (c // nx) % ny] + ([c // (nx * ny)] if self.dim == 3 else [])
                cell, off = np.stack(coords).astype(np.int32), st["off"]
            else:
                cell, off = np.zeros((self.dim, n), np.int32), np.zeros((self.dim, n))
            p = Particles(q=rec["q"], m=rec["m"], cell=cell, off=off, u=st["u"], w=st["w"], id=st["id"])
            sp = Species(self, rec["q"], rec["m"], rec["cap"])
            sp.upload(p, True, stream, rec["max_weight"])
            if self.precision == FP64:
                # the positions themselves, not rebuilt from cell + offset
                v = sp._views(0)
                for d in range(self.dim):
                    v["x"][d][:n] = torch.from_numpy(st["x"][d]).to(self.device)
            self.species.append(sp)
            sp.set_next_id(rec["next_id"], stream)
        if self.precision == FP32_FIXED and self.info().fixed_shift != ckpt["fixed_shift"]:
            raise ValueError("restored species give another fixed-point shift (capacities differ)")
        for name in ("E", "B", "J"):
            for dst, src in zip(getattr(self, name), ckpt[name]):
                dst.copy_(torch.from_numpy(src).to(self.device))
        torch.cuda.synchronize(self.device)

    def qed_init(self, eps_ref, seed, stream=None):
        """Build the emission tables; eps_ref = hbar omega / (m c^2) of the unit frequency."""
        _check(load().lpic_qed_init(self.h_, float(eps_ref), int(seed) & (2**64 - 1), _stream(stream)))

    def qed_initial_tau(self, n_ids, stream=None, photons=False) -> torch.Tensor:
        """Optical depths -ln r for ids 0..n_ids-1 (float32 device tensor);
        photons=True: the pair-creation depths of photons."""
        tau = torch.empty(max(int(n_ids), 1), dtype=torch.float32, device=self.device)
        _check(load().lpic_qed_initial_tau(self.h_, tau.data_ptr(), int(n_ids), int(bool(photons)),
                                           _stream(stream)))
        return tau[: int(n_ids)]

    def qed_compton(self, electrons, photons, tau, step, stream=None, photon_tau=None):
        """One emission pass of `electrons` into `photons` (Species objects);
        photon_tau (optional) receives the new photons' pair-creation depths."""
        assert tau.dtype == torch.float32 and tau.is_cuda and tau.is_contiguous()
        pt, pn = (None, 0) if photon_tau is None else (photon_tau.data_ptr(), photon_tau.numel())
        if photon_tau is not None:
            assert photon_tau.dtype == torch.float32 and photon_tau.is_cuda and photon_tau.is_contiguous()
        _check(load().lpic_qed_compton(self.h_, electrons.id, photons.id, tau.data_ptr(), tau.numel(),
                                       pt, pn, int(step), _stream(stream)))

    def qed_fuse(self, electrons, photons, tau, first_step=0, stream=None, photon_tau=None):
        """Emission of `electrons` into `photons` inside every push of
        `electrons` (photons=None turns it off); the counter word starts at
        first_step and advances with each full step."""
        if photons is None:
            _check(load().lpic_qed_fuse(self.h_, electrons.id, -1, None, 0, None, 0, 0, _stream(stream)))
            return
        assert tau.dtype == torch.float32 and tau.is_cuda and tau.is_contiguous()
        pt, pn = (None, 0) if photon_tau is None else (photon_tau.data_ptr(), photon_tau.numel())
        if photon_tau is not None:
            assert photon_tau.dtype == torch.float32 and photon_tau.is_cuda and photon_tau.is_contiguous()
        _check(load().lpic_qed_fuse(self.h_, electrons.id, photons.id, tau.data_ptr(), tau.numel(), pt, pn,
                                    int(first_step), _stream(stream)))

    def qed_set_step(self, step, stream=None):
        _check(load().lpic_qed_set_step(self.h_, int(step), _stream(stream)))

    def qed_breit_wheeler(self, photons, electrons, positrons, tau, step, stream=None):
        """One pair-creation pass of `photons` into `electrons` and `positrons`."""
        assert tau.dtype == torch.float32 and tau.is_cuda and tau.is_contiguous()
        _check(load().lpic_qed_breit_wheeler(self.h_, photons.id, electrons.id, positrons.id, tau.data_ptr(),
                                             tau.numel(), int(step), _stream(stream)))

    def qed_pair_eval(self, chi, r, stream=None):
        """Device pair-table lookups: (H(chi), eta(chi, r)) as float64 numpy arrays."""
        c = torch.as_tensor(np.asarray(chi, np.float64), device=self.device).contiguous()
        rr = torch.as_tensor(np.asarray(r, np.float64), device=self.device).contiguous()
        h, eta = torch.empty_like(c), torch.empty_like(c)
        _check(load().lpic_qed_pair_eval(self.h_, c.data_ptr(), rr.data_ptr(), c.numel(), h.data_ptr(),
                                         eta.data_ptr(), _stream(stream)))
        torch.cuda.synchronize(self.device)
        return h.cpu().numpy(), eta.cpu().numpy()

    def qed_eval(self, chi, r, stream=None):
        """Device table lookups: (h(chi), xi(chi, r)) as float64 numpy arrays."""
        c = torch.as_tensor(np.asarray(chi, np.float64), device=self.device).contiguous()
        rr = torch.as_tensor(np.asarray(r, np.float64), device=self.device).contiguous()
        assert c.shape == rr.shape
        h = torch.empty_like(c)
        xi = torch.empty_like(c)
        _check(load().lpic_qed_eval(self.h_, c.data_ptr(), rr.data_ptr(), c.numel(), h.data_ptr(),
                                    xi.data_ptr(), _stream(stream)))
        torch.cuda.synchronize(self.device)
        return h.cpu().numpy(), xi.cpu().numpy()

    def info(self) -> GridInfo:
        out = GridInfo()
        _check(load().lpic_grid_get_info(self.h_, ctypes.byref(out)))
        return out

    # -- the path
    def maxwell_half(self, half, t=0.0, stream=None):
        _check(load().lpic_maxwell_half_step(self.h_, half, t, _stream(stream)))

    def zero_current(self, stream=None):
        _check(load().lpic_zero_current(self.h_, _stream(stream)))

    def sort(self, sid=-1, stream=None):
        _check(load().lpic_sort_particles(self.h_, sid, _stream(stream)))

    def gather_push_deposit(self, sid, stream=None):
        _check(load().lpic_gather_push_deposit(self.h_, sid, _stream(stream)))

    def step(self, t, stream=None):
        _check(load().lpic_step(self.h_, t, _stream(stream)))

    def set_clock(self, t, stream=None):
        _check(load().lpic_set_clock(self.h_, t, _stream(stream)))

    def graph_steps(self, nsteps, stream=None):
        """nsteps full steps replayed from captured CUDA graphs (device clock)."""
        _check(load().lpic_graph_steps(self.h_, nsteps, _stream(stream)))

    def kernel_timing(self, max_launches):
        """Record CUDA events around the next max_launches fused-kernel launches."""
        _check(load().lpic_kernel_timing(self.h_, int(max_launches)))

    def kernel_time(self):
        """(summed milliseconds, launches) of the timed fused-kernel launches."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _check(load().lpic_kernel_time(self.h_, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def diagnostics(self, stream=None) -> Diag:
        out = Diag()
        _check(load().lpic_diagnostics(self.h_, ctypes.byref(out), _stream(stream)))
        return out

    def check_status(self, stream=None) -> int:
        bits = ctypes.c_uint()
        rc = load().lpic_check_status(self.h_, _stream(stream), ctypes.byref(bits))
        if rc not in (0, 4):
            _check(rc)
        return bits.value

    def gather_fields(self, sid, out=None, stream=None) -> torch.Tensor:
        """Unfused stage 1: the species' particles' fields, float32 (6, capacity)."""
        sp = self.species[sid]
        if out is None:
            out = torch.empty((6, sp.cap), dtype=torch.float32, device=self.device)
        _check(load().lpic_gather_fields(self.h_, sid, out.data_ptr(), _stream(stream)))
        return out

    def push_deposit_fields(self, sid, fields, stream=None):
        """Unfused stage 2: push and deposit with the given per-particle fields."""
        assert fields.dtype == torch.float32 and fields.is_contiguous()
        assert fields.shape == (6, self.species[sid].cap)
        _check(load().lpic_push_deposit_fields(self.h_, sid, fields.data_ptr(), _stream(stream)))

    def step_resolved(self, t, sid, aux: "Grid", stream=None):
        """One step that also advances aux with the current of species sid alone."""
        _check(load().lpic_step_resolved(self.h_, t, sid, aux.h_, _stream(stream)))

    def div_e(self, stream=None) -> torch.Tensor:
        """Discrete divergence of E at the integer nodes (float64)."""
        out = torch.empty(self.field_shape, dtype=torch.float64, device=self.device)
        _check(load().lpic_div_e(self.h_, out.data_ptr(), _stream(stream)))
        return out

    def rho(self, stream=None) -> torch.Tensor:
        """Charge density of all species' stored positions (float64, field units)."""
        inf = self.info() if self.precision != FP64 else None
        tot = torch.zeros(self.field_shape, dtype=torch.float64, device=self.device)
        for sp in self.species:
            r = sp.charge(stream)
            tot += r if inf is None else r.to(torch.float64) * inf.rho_scale
        return tot

    def current(self) -> list:
        """J as float64 in field units (FP32 path: J_int * j_scale)."""
        if self.precision == FP64:
            return [j.clone() for j in self.J]
        inf = self.info()
        return [self.J[c].to(torch.float64) * inf.j_scale[c] for c in range(3)]


class Ensemble:
    """Independent grids stepped together (batched kernels, one persistent
    particle kernel with a device work queue)."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h_.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(load().lpic_create_ensemble(arr, len(self.grids), ctypes.byref(h)))
        self.h_ = h

    def close(self):
        if getattr(self, "h_", None):
            load().lpic_destroy_ensemble(self.h_)
            self.h_ = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, stream=None):
        _check(load().lpic_ensemble_step(self.h_, _stream(stream)))

    def graph_steps(self, nsteps, stream=None):
        _check(load().lpic_ensemble_graph_steps(self.h_, int(nsteps), _stream(stream)))

    def check_status(self, stream=None) -> int:
        bits = ctypes.c_uint()
        rc = load().lpic_ensemble_check_status(self.h_, _stream(stream), ctypes.byref(bits))
        if rc not in (0, 4):
            _check(rc)
        return bits.value

    def launches(self) -> int:
        n = ctypes.c_longlong()
        _check(load().lpic_ensemble_launches(self.h_, ctypes.byref(n)))
        return n.value


def debug_fail_alloc(nth: int):
    """Tests: make the library's nth device allocation from now fail (0: off)."""
    _check(load().lpic_debug_fail_alloc(int(nth)))


def grid_for(wl, precision=None, tile=None, device="cuda", block_particles=0, sort_interval=0,
             maxwell_fp64=False) -> Grid:
    """A Grid for a workloads.Workload (laser centred transversally);
    maxwell_fp64 keeps FP64 master fields on the FP32 path."""
    from . import workloads as W
    prec = precision if precision is not None else (FP64 if wl.precision == "fp64" else FP32_FIXED)
    laser = None
    if wl.laser is not None:
        c = wl.laser_center()
        laser = W.LaserSpec(wl.laser.a0, wl.laser.w0, wl.laser.tau, wl.laser.omega)
        laser.yc, laser.zc = c[0], (c[1] if wl.dim == 3 else 0.0)
    pml = PmlSpec() if getattr(wl, "boundary", "mur") == "cpml" else None
    return Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, prec, wl.absorb_x, laser, tile, device,
                block_particles, sort_interval, pml, maxwell_fp64)


def save_checkpoint(G: Grid, path, stream=None):
    """Grid.checkpoint() written to an .npz file."""
    ck = G.checkpoint(stream)
    flat = {"meta": np.array([ck["dim"], ck["precision"], ck.get("fixed_shift", 0), len(ck["species"])]),
            "n": np.array(ck["n"])}
    for name in ("E", "B", "J"):
        for c, a in enumerate(ck[name]):
            flat[f"{name}{c}"] = a
    for k, rec in enumerate(ck["species"]):
        flat[f"s{k}_scalars"] = np.array([rec["q"], rec["m"], rec["cap"], rec["max_weight"], rec["next_id"]],
                                         dtype=np.float64)
        for key, a in rec["particles"].items():
            flat[f"s{k}_{key}"] = a
    np.savez(path, **flat)


def load_checkpoint(G: Grid, path, stream=None):
    """Restore an .npz written by save_checkpoint into a fresh grid G."""
    z = np.load(path)
    dim, prec, fshift, ns = (int(v) for v in z["meta"])
    ck = {"dim": dim, "precision": prec, "fixed_shift": fshift, "n": list(z["n"]),
          "E": [z[f"E{c}"] for c in range(3)], "B": [z[f"B{c}"] for c in range(3)],
          "J": [z[f"J{c}"] for c in range(3)], "species": []}
    keys = ("cell", "off", "u", "w", "id") if prec == FP32_FIXED else ("x", "u", "w", "id")
    for k in range(ns):
        q, m, cap, wmax, nid = z[f"s{k}_scalars"]
        ck["species"].append({"q": q, "m": m, "cap": int(cap), "max_weight": wmax, "next_id": int(nid),
                              "particles": {key: z[f"s{k}_{key}"] for key in keys}})
    G.restore(ck, stream)
