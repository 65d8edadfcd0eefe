"""Host-side checks of the synthetic QED set-up (pair plasma for the
emission and pair-creation passes): photon-energy unit of the laser
wavelength, identical lepton positions, ids unique across the emitting
species (the emission draws are keyed by id), and the temperature of the
Maxwell-Juttner momenta."""
import math

import numpy as np

from paper_2607_13507_b300 import workloads as W


def test_qed2d_units_and_species():
    wl = W.qed2d(n=16, ppc=4)
    # hbar omega / (m c^2) of a 0.8 um wavelength: 1.5498 eV / 510999 eV
    assert abs(wl.qed_eps_ref / (1.239841984 / 0.8 / 510998.95) - 1.0) < 1e-4
    assert wl.b0 == 4.0 and wl.dim == 2 and not wl.absorb_x
    assert abs(wl.h[0] - 2.0 * math.pi / 32) < 1e-15
    e, p = W.load_all(wl)
    assert e.q == -1.0 and p.q == 1.0 and e.m == p.m == 1.0
    assert e.n == p.n == 16 * 16 * 4
    assert np.array_equal(e.cell, p.cell) and np.array_equal(e.off, p.off)
    ids = np.concatenate([e.id, p.id])
    assert len(np.unique(ids)) == ids.size and ids.min() == 0 and ids.max() == ids.size - 1


def test_qed2d_temperature():
    theta = 3000.0
    e, _ = W.load_all(W.qed2d(n=32, ppc=16, theta=theta))
    u = e.u.astype(np.float64)
    gam = np.sqrt(1.0 + (u ** 2).sum(0))
    # Maxwell-Juttner: <gamma> = 3 theta + K1(1/theta) / K2(1/theta), and the
    # Bessel ratio is about 1 / (2 theta) here; the std of gamma is sqrt(3) theta
    assert abs(gam.mean() - 3.0 * theta) < 5.0 * math.sqrt(3.0) * theta / math.sqrt(gam.size) + 1.0
    # pressure: <u^2 / gamma> = 3 theta
    p = (u ** 2).sum(0) / gam
    assert abs(p.mean() / (3.0 * theta) - 1.0) < 5.0 * p.std() / p.mean() / math.sqrt(p.size)
