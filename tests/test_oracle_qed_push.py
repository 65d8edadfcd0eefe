"""Pins of the oracle's particle loop with nonlinear Compton emission inside
it (Algorithm 1: the QED events sit between the field interpolation and the
momentum push; Sec. 3.4 for the event itself), in uniform fields, where the
interpolated fields are the fields themselves:

* with a depth that cannot run out, the loop equals the plain push bit for
  bit (positions, momenta, current), and the depth falls by W dt with W the
  photon rate of the spectrum integrated here with scipy, at the chi that
  u^n (not u^{n+1}) gives in the closed form for uniform fields;
* with a depth that runs out at once, every particle emits: the photon
  carries k = xi gamma^n along u^n, xi inverting the spectrum's cumulative
  (scipy quadrature) at the first Philox word of counter (p, step, 0, 0);
  the particle's pushed momentum is the Boris push of u^n - k u^n/|u^n|
  (recoil first), the photon starts at x^{n+1/2} and is stored half a step
  later along its direction, the depth restarts at -ln of the second word;
* a particle moving along B with no E (chi = 0) never emits.

No GPU is needed.
"""
import math

import numpy as np
from scipy import integrate, special

from oracle import oracle as O

ALPHA = 1.0 / 137.035999084
SEED = 0x5EED0F0B
EPS = 2e-6


def _spectrum(xi, chi):
    """S(xi, chi) with scipy's Bessel functions."""
    if xi <= 0.0 or xi >= 1.0:
        return 0.0
    d = 2.0 * xi / (3.0 * chi * (1.0 - xi))
    if d > 600.0:
        return 0.0
    tail = integrate.quad(lambda s: special.kv(1.0 / 3.0, s), d, d + 60.0, limit=200)[0]
    return (1.0 - xi + 1.0 / (1.0 - xi)) * special.kv(2.0 / 3.0, d) - tail


def _h(chi):
    top = min(1.0, 60.0 * chi)
    return integrate.quad(lambda x: _spectrum(x, chi), 0.0, top, limit=400, points=[min(chi, 0.5 * top)])[0]


def _chi(u, E, B):
    gam = math.sqrt(1.0 + u @ u)
    b = u / gam
    f = E + np.cross(b, B)
    return EPS * gam * math.sqrt(max(f @ f - (b @ E) ** 2, 0.0))


def _setup(n=6, seed=3):
    wl_n, h, dt = (16, 16), (0.5, 0.5), 0.25
    g = O.Grid(2, wl_n, h, dt, 1)
    E0 = np.array([150.0, -420.0, 80.0])
    B0 = np.array([60.0, 210.0, 600.0])
    for c in range(3):
        g.E[c][...] = E0[c]
        g.B[c][...] = B0[c]
    rng = np.random.Generator(np.random.Philox(seed))
    x = rng.uniform(1.0, 7.0, size=(2, n))
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    u = d * np.exp(rng.uniform(np.log(20.0), np.log(200.0), n))
    w = rng.uniform(0.5, 2.0, n)
    return g, E0, B0, x, u, w


def _uniform(n):
    """(x + 1/2) 2^-32 of the Philox words of counter (p, step, 0, 0)."""
    return lambda p, step: [(v + 0.5) / 2.0 ** 32 for v in O.philox([p, step, 0, 0], [SEED & 0xFFFFFFFF, SEED >> 32])]


def test_no_event_equals_plain_push_and_depth_falls_by_the_rate():
    g, E0, B0, x, u, w = _setup()
    n = x.shape[1]
    a = O.Species(-1.0, 1.0, x, u.copy(), w.copy())
    b = O.Species(-1.0, 1.0, x, u.copy(), w.copy())
    O.push_species(g, a)
    Ja = [j.copy() for j in g.J]
    for c in range(3):
        g.J[c][...] = 0.0
    tau = np.full(n, 1e6)
    ph, owner = O.push_species_qed(g, b, EPS, SEED, 7, tau)
    assert ph.x.shape[1] == 0 and owner.size == 0
    assert np.array_equal(a.x, b.x) and np.array_equal(a.u, b.u)
    for c in range(3):
        assert np.array_equal(Ja[c], g.J[c])
    worst_other = 0.0
    for p in range(n):
        chi = _chi(u[:, p], E0, B0)
        gam = math.sqrt(1.0 + u[:, p] @ u[:, p])
        W = ALPHA / (EPS * math.sqrt(3.0) * math.pi * gam) * _h(chi)
        assert abs((1e6 - tau[p]) / (W * g.dt) - 1.0) < 1e-3, (p, chi)
        # the rate at u^{n+1} (emission after the push) would differ
        gam1 = math.sqrt(1.0 + a.u[:, p] @ a.u[:, p])
        W1 = ALPHA / (EPS * math.sqrt(3.0) * math.pi * gam1) * _h(_chi(a.u[:, p], E0, B0))
        worst_other = max(worst_other, abs(W1 / W - 1.0))
    assert worst_other > 2e-2


def test_every_particle_emits_with_recoil_before_the_push():
    g, E0, B0, x, u, w = _setup(n=5, seed=4)
    n = x.shape[1]
    sp = O.Species(-1.0, 1.0, x, u.copy(), w.copy())
    tau = np.full(n, 1e-300)
    step = 11
    ph, owner = O.push_species_qed(g, sp, EPS, SEED, step, tau)
    assert sorted(owner.tolist()) == list(range(n))
    draw = _uniform(n)
    L = np.array([16 * 0.5, 16 * 0.5])
    for j, p in enumerate(owner):
        r1, r2 = draw(int(p), step)[:2]
        un = u[:, p]
        gam = math.sqrt(1.0 + un @ un)
        umag = math.sqrt(un @ un)
        chi = _chi(un, E0, B0)
        k = np.linalg.norm(ph.u[:, j])
        xi = k / gam
        # xi inverts the normalised cumulative of S at r1
        top = min(1.0, 60.0 * chi)
        cum = integrate.quad(lambda s: _spectrum(s, chi), 0.0, xi, limit=400, points=[min(chi, 0.5 * xi)])[0]
        assert abs(cum / _h(chi) - r1) < 2e-3, (p, cum / _h(chi), r1, top)
        # the photon moves along u^n with the emitter's weight
        assert np.allclose(ph.u[:, j] / k, un / umag, rtol=0, atol=1e-14)
        assert ph.w[j] == w[p]
        # recoil first, then the momentum push in the fields at x^{n+1/2}
        ur = un * (1.0 - k / umag)
        expect = O.boris(-1.0, 1.0, g.dt, ur, E0, B0)
        assert np.allclose(sp.u[:, p], expect, rtol=1e-13, atol=0)
        assert np.allclose(ur + ph.u[:, j], un, rtol=1e-13, atol=0)
        # the photon leaves x^{n+1/2} and is stored half a step later
        xh = x[:, p] + 0.5 * g.dt * un[:2] / gam
        xp = np.remainder(xh + 0.5 * g.dt * un[:2] / umag, L)
        assert np.allclose(ph.x[:2, j], xp, rtol=0, atol=1e-13)
        assert abs(tau[p] + math.log(r2)) < 1e-12


def test_no_emission_without_a_transverse_force():
    g, E0, B0, x, u, w = _setup(n=3, seed=5)
    # no E, momenta along B: beta x B = 0 (a longitudinal E would still give
    # chi = eps_ref |E|)
    for c in range(3):
        g.E[c][...] = 0.0
        g.B[c][...] = 0.0
    g.B[2][...] = 700.0
    u = np.zeros_like(u)
    u[2] = [200.0, -50.0, 900.0]
    sp = O.Species(-1.0, 1.0, x, u.copy(), w.copy())
    tau = np.full(3, 1e-300)
    ph, owner = O.push_species_qed(g, sp, EPS, SEED, 0, tau)
    assert owner.size == 0
    assert np.all(tau == 1e-300)
