"""Pins of the oracle's nonlinear Compton module (Sec. 3.4) against
independent facts:

* Philox4x32-10 reproduces the published known-answer vectors;
* the modified Bessel integrals match scipy's K_nu and its quadrature;
* in the classical limit chi -> 0 the photon number rate tends to
  5 alpha chi / (2 sqrt(3) gamma) (per unit time, m c^2 / hbar units) and
  the radiated power to (2/3) alpha chi^2 (the Larmor power), both from the
  spectrum S integrated here with scipy, independently of the oracle's own
  integration;
* the sampled photon energy fraction inverts the spectrum's CDF;
* chi_e has its closed forms, and an emission conserves momentum.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O

ALPHA = 1.0 / 137.035999084


def test_philox_known_answers():
    assert O.philox([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert O.philox([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


@pytest.mark.parametrize("x", [0.003, 0.1, 1.0, 5.0, 20.0])
def test_bessel_integrals(x):
    for nu in (1.0 / 3.0, 2.0 / 3.0):
        assert abs(O.bessel_k(nu, x) / special.kv(nu, x) - 1.0) < 1e-10
    ref = integrate.quad(lambda s: special.kv(1.0 / 3.0, s), x, x + 60.0, limit=200)[0]  # K decays as e^-s
    assert abs(O.bessel_k_int(1.0 / 3.0, x) / ref - 1.0) < 1e-7


def _scipy_moment(chi, k):
    """int_0^1 xi^k S(xi, chi) dxi with scipy's Bessel functions."""
    def S(xi):
        d = 2.0 * xi / (3.0 * chi * (1.0 - xi))
        ik = integrate.quad(lambda s: special.kv(1.0 / 3.0, s), d, math.inf, limit=200)[0]
        return (1.0 - xi + 1.0 / (1.0 - xi)) * special.kv(2.0 / 3.0, d) - ik
    # xi = y^3 removes the xi^(-2/3) end point behaviour
    return integrate.quad(lambda y: S(y ** 3) * 3.0 * y ** 2 * y ** (3 * k), 0.0, 1.0 - 1e-12, limit=400)[0]


def test_classical_limits():
    chi, gam, eps = 1e-4, 50.0, 1e-3
    pref = ALPHA / (eps * math.sqrt(3.0) * math.pi * gam)
    # number rate: the oracle's integration and the closed form
    W = O.compton_rate(chi, gam, eps)
    assert abs(W / (5.0 * ALPHA * chi / (2.0 * math.sqrt(3.0) * gam * eps)) - 1.0) < 2e-3
    # the spectrum's moments with scipy: number and power (xi gamma m c^2 per photon)
    n0 = pref * _scipy_moment(chi, 0)
    assert abs(n0 / W - 1.0) < 1e-3
    p1 = pref * gam * _scipy_moment(chi, 1)
    assert abs(p1 / (2.0 / 3.0 * ALPHA * chi ** 2 / eps) - 1.0) < 2e-3


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0])
def test_sampled_fraction_inverts_the_spectrum(chi):
    def S(xi):
        if xi <= 0.0 or xi >= 1.0:
            return 0.0
        return O.compton_s(xi, chi)
    tot = integrate.quad(lambda y: S(y ** 3) * 3 * y * y, 0, 1, limit=400)[0]
    for r in (0.1, 0.5, 0.9):
        xi = O.compton_xi(chi, r)
        part = integrate.quad(lambda y: S(y ** 3) * 3 * y * y, 0, xi ** (1 / 3), limit=400)[0]
        assert abs(part / tot - r) < 2e-3


def test_chi_closed_forms():
    eps = 1e-3
    u = np.array([30.0, 0.0, 0.0])
    B = np.array([0.0, 0.0, 200.0])
    assert abs(O.chi_e(u, np.zeros(3), B, eps) / (eps * 30.0 * 200.0) - 1.0) < 1e-12
    # a particle moving along E feels E / gamma^0: chi = eps E
    E = np.array([50.0, 0.0, 0.0])
    assert abs(O.chi_e(u, E, np.zeros(3), eps) / (eps * 50.0) - 1.0) < 1e-12


def test_emission_conserves_momentum():
    nx, ny, dx = 16, 16, 0.1
    dt = 0.95 * dx / math.sqrt(2)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1)
    g.B[2][...] = 300.0
    n = 200
    rng = np.random.Generator(np.random.Philox(3))
    x = rng.uniform(0, nx * dx, (2, n))
    u = np.zeros((3, n))
    u[0] = 40.0
    sp = O.Species(-1.0, 1.0, x, u, np.full(n, 1e-9))
    tau = np.full(n, 1e-9)                   # every particle emits now
    p0 = sp.u.copy()
    ph = O.qed_compton(g, sp, 1e-3, 7, 1, tau)
    assert ph.n == n
    assert np.allclose(sp.u + ph.u, p0, rtol=0, atol=1e-9)
    assert np.all(tau > 0)


def test_large_chi_asymptote_of_the_rate():
    # chi -> inf: delta -> 0 over the bulk of xi, K_{2/3}(delta) -> Gamma(2/3) (delta/2)^{-2/3} / 2
    # and the K_{1/3} tail stays finite, so int S dxi -> Gamma(2/3) (3 chi)^{2/3}
    # (B(1/3, 8/3) + B(1/3, 2/3)) / 2, approached like 1 - a chi^{-2/3}
    c = 0.5 * special.gamma(2.0 / 3.0) * 3.0 ** (2.0 / 3.0) * (special.beta(1.0 / 3.0, 8.0 / 3.0)
                                                                  + special.beta(1.0 / 3.0, 2.0 / 3.0))

    def ratio(chi):
        h = O.compton_rate(chi, 1.0, 1.0) * math.sqrt(3.0) * math.pi / ALPHA
        return h / (c * chi ** (2.0 / 3.0))

    r2, r3 = ratio(1e2), ratio(1e3)
    assert 0.0 < 1.0 - r3 < 1.0 - r2 < 0.05
    assert abs((1.0 - r3) - (1.0 - r2) * 10.0 ** (-2.0 / 3.0)) < 2e-3
