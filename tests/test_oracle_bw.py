"""Pins of the oracle's Breit-Wheeler pair creation (Sec. 3.4) against what
the mathematics fixes: the small-chi asymptote of the pair rate (Laplace's
method on the spectrum: W -> (3 sqrt(3) / (16 sqrt(2))) alpha chi / (eps k)
exp(-8 / (3 chi))), the spectrum against scipy's Bessel functions, its
symmetry between electron and positron, the inverse cumulative against scipy
quadrature, closed forms of chi_gamma, and the kinematics of an event."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O

ALPHA = 1.0 / 137.035999084


def _asym(chi, k, eps):
    return 3.0 * math.sqrt(3.0) / (16.0 * math.sqrt(2.0)) * ALPHA * chi / (eps * k) * math.exp(-8.0 / (3.0 * chi))


def test_small_chi_asymptote():
    # corrections are O(chi): the ratio extrapolated linearly to chi = 0 is 1
    r1 = O.bw_rate(0.01, 100.0, 1e-3) / _asym(0.01, 100.0, 1e-3)
    r2 = O.bw_rate(0.02, 100.0, 1e-3) / _asym(0.02, 100.0, 1e-3)
    assert abs(r1 - 1.0) < 5e-3
    assert abs(2.0 * r1 - r2 - 1.0) < 2e-4
    # W scales as 1 / (eps k)
    assert abs(O.bw_rate(0.5, 10.0, 1e-3) / O.bw_rate(0.5, 40.0, 4e-3) - 16.0) < 1e-9


def _f_scipy(eta, chi):
    z = 2.0 / (3.0 * chi * eta * (1.0 - eta))
    ik = integrate.quad(lambda s: special.kv(1.0 / 3.0, s), z, z + 60.0, limit=200)[0]
    return (eta / (1.0 - eta) + (1.0 - eta) / eta) * special.kv(2.0 / 3.0, z) + ik


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0, 200.0])
def test_spectrum_against_scipy_and_symmetric(chi):
    for eta in (0.05, 0.2, 0.5, 0.8):
        ref = _f_scipy(eta, chi)
        assert abs(O.bw_f(eta, chi) / ref - 1.0) < 1e-7
        assert abs(O.bw_f(eta, chi) - O.bw_f(1.0 - eta, chi)) <= 1e-12 * ref


@pytest.mark.parametrize("chi", [0.3, 3.0, 50.0])
def test_sampled_share_inverts_the_spectrum(chi):
    tot = integrate.quad(lambda e: _f_scipy(e, chi), 1e-9, 1 - 1e-9, limit=400, points=[0.5])[0]
    for r in (0.05, 0.3, 0.5, 0.9):
        eta = O.bw_eta(chi, r)
        part = integrate.quad(lambda e: _f_scipy(e, chi), 1e-9, eta, limit=400)[0]
        assert abs(part / tot - r) < 1e-3
        assert abs(O.bw_eta(chi, r) + O.bw_eta(chi, 1.0 - r) - 1.0) < 1e-3
    assert abs(O.bw_eta(chi, 0.5) - 0.5) < 1e-9


def test_chi_gamma_closed_forms():
    eps = 1e-3
    k = np.array([500.0, 0.0, 0.0])
    assert abs(O.chi_g(k, np.zeros(3), np.array([0.0, 0.0, 80.0]), eps) / (eps * 500.0 * 80.0) - 1.0) < 1e-12
    # along E, and in a plane wave co-moving with the photon: no pairs
    assert O.chi_g(k, np.array([30.0, 0.0, 0.0]), np.zeros(3), eps) == 0.0
    assert O.chi_g(k, np.array([0.0, 30.0, 0.0]), np.array([0.0, 0.0, 30.0]), eps) == 0.0
    # counter-propagating plane wave: chi = 2 eps k E
    kb = -k
    assert abs(O.chi_g(kb, np.array([0.0, 30.0, 0.0]), np.array([0.0, 0.0, 30.0]), eps) / (2 * eps * 500 * 30) - 1) < 1e-12


def test_initial_depth_kinds():
    ids = np.arange(50)
    assert np.array_equal(O.qed_initial_tau_kind(ids, 2, 99), O.qed_initial_tau(ids, 99))
    assert not np.allclose(O.qed_initial_tau_kind(ids, 3, 99), O.qed_initial_tau(ids, 99))


def test_pair_event_kinematics():
    nx, ny, dx = 16, 16, 0.1
    dt = 0.95 * dx / math.sqrt(2)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1)
    g.B[2][...] = 400.0
    n = 100
    rng = np.random.Generator(np.random.Philox(5))
    x = rng.uniform(0, nx * dx, (2, n))
    u = np.zeros((3, n))
    u[0] = np.where(np.arange(n) < 10, 1.5, 2000.0)      # the first ten below threshold
    ph = O.Species(0.0, 0.0, x, u, np.full(n, 2e-9))
    tau = np.full(n, -1.0)                                 # every eligible photon converts now
    el, po = O.qed_bw(g, ph, 1e-3, 7, 4, tau)
    assert el.n == po.n == n - 10
    assert np.array_equal(ph.alive[:10], np.ones(10)) and not ph.alive[10:].any()
    assert np.allclose(el.u + po.u, u[:, 10:], rtol=0, atol=1e-12)
    assert np.all(el.u[0] > 0) and np.all(po.u[0] > 0)
    assert np.array_equal(el.x[:2], x[:, 10:]) and np.array_equal(el.w, ph.w[10:])
    eta = el.u[0] / 2000.0
    assert 0.3 < eta.mean() < 0.7


def test_large_chi_asymptote():
    # chi -> inf: z -> 0 over the bulk of eta, K_{2/3}(z) -> Gamma(2/3) (z/2)^{-2/3} / 2 and
    # the K_{1/3} tail stays finite, so int F deta -> Gamma(2/3) (3 chi)^{2/3} B(8/3, 2/3),
    # approached like 1 - a chi^{-2/3}
    c = special.gamma(2.0 / 3.0) * 3.0 ** (2.0 / 3.0) * special.beta(8.0 / 3.0, 2.0 / 3.0)

    def ratio(chi):
        H = O.bw_rate(chi, 10.0, 1.0) * 10.0 * math.sqrt(3.0) * math.pi / ALPHA
        return H / (c * chi ** (2.0 / 3.0))

    r2, r3 = ratio(1e2), ratio(1e3)
    assert 0.0 < 1.0 - r3 < 1.0 - r2 < 0.1
    assert abs((1.0 - r3) - (1.0 - r2) * 10.0 ** (-2.0 / 3.0)) < 2e-3
