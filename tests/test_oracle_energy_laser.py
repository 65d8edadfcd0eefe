"""Pins of the oracle's energy diagnostic (Sec. 4.1) and of its incoming
laser (Sec. 4.2) against what the definitions fix, independently of the
formulas inside the oracle:

* kinetic energy sum w m (gamma - 1) on momenta with rational gamma
  (u = 3/4 gives gamma = 5/4 exactly), photons w |u|, total charge sum q w;
* field energy (1/2) sum (E^2 + B^2) dV of sinusoidal fields, whose discrete
  sums of sin^2 and cos^2 over whole periods are N / 2 (orthogonality);
* a cold Langmuir oscillation hands its energy from the particles to E_x and
  back: the two maxima agree and their sum stays constant (a dropped 1/2, a
  dropped dV or gamma in place of gamma - 1 breaks either);
* the laser is measured on the grid after it has entered through the x-min
  edge: amplitude a0 at the centre of the sin^2 envelope, half of it at a
  quarter of the duration, nothing before and after the duration, carrier
  frequency omega and a transverse 1/e radius w0 of the envelope (2D and 3D).

No GPU is needed.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


# ---------------------------------------------------------------- kinetic energy
def test_kinetic_energy_and_charge_closed_forms():
    g = O.Grid(2, (4, 4), (0.5, 0.25), 0.1, 1)
    # gamma = 5/4 (u = 3/4), 13/5 (u = 12/5), 17/15 (u = 8/15): rational energies
    u = np.array([[0.75, 0.0, 0.0], [0.0, 2.4, 0.0], [0.0, 0.0, -8.0 / 15.0]]).T
    x = np.array([[0.1, 0.2], [0.7, 0.3], [1.1, 0.9]]).T
    w = np.array([2.0, 0.5, 3.0])
    e = O.Species(-1.0, 1.0, x, u, w)
    p = O.Species(1.0, 1836.0, x, u, w)
    ek, ef, qt = O.energy(g, [e, p])
    gm1 = np.array([0.25, 1.6, 2.0 / 15.0])
    expect = float(np.sum(w * gm1)) * (1.0 + 1836.0)
    assert abs(ek - expect) < 1e-14 * expect
    assert ef == 0.0
    assert abs(qt - (-w.sum() + w.sum())) < 1e-15
    ek1, _, qt1 = O.energy(g, [e])
    assert abs(ek1 - float(np.sum(w * gm1))) < 1e-15 * ek1
    assert abs(qt1 + w.sum()) < 1e-15
    # removed particles carry nothing
    e2 = O.Species(-1.0, 1.0, x, u, w, alive=[1, 0, 1])
    assert abs(O.energy(g, [e2])[0] - (2.0 * 0.25 + 3.0 * 2.0 / 15.0)) < 1e-15
    # photons (m = 0) carry w |u|: |(3, 4, 0)| = 5, |(2, 3, 6)| = 7
    ph = O.Species(0.0, 0.0, x[:, :2], np.array([[3.0, 4.0, 0.0], [2.0, 3.0, 6.0]]).T, [1.5, 0.25])
    assert abs(O.energy(g, [ph])[0] - (7.5 + 1.75)) < 1e-14


# ---------------------------------------------------------------- field energy
@pytest.mark.parametrize("dim", [2, 3])
def test_field_energy_of_sinusoids(dim):
    n = (12, 10, 8)[:dim]
    h = (0.3, 0.2, 0.5)[:dim]
    g = O.Grid(dim, n, h, 0.05, 1)
    shape = g.E[0].shape                       # (nz, ny, nx)
    k = np.arange(shape[0]).reshape(-1, 1, 1)
    j = np.arange(shape[1]).reshape(1, -1, 1)
    i = np.arange(shape[2]).reshape(1, 1, -1)
    A = [0.7, -1.3, 0.4]
    C = [2.0, 0.6, -0.9]
    ones = np.ones(shape)
    g.E[0][...] = A[0] * np.sin(2 * math.pi * 3 * i / n[0]) * ones
    g.E[1][...] = A[1] * np.cos(2 * math.pi * 2 * j / n[1]) * ones
    g.E[2][...] = A[2] * ones                                   # constant: sum = N
    g.B[0][...] = C[0] * np.cos(2 * math.pi * 1 * i / n[0]) * ones
    g.B[1][...] = C[1] * np.sin(2 * math.pi * 4 * j / n[1]) * ones
    if dim == 3:
        g.B[2][...] = C[2] * np.sin(2 * math.pi * 3 * k / n[2]) * ones
    else:
        g.B[2][...] = C[2] * np.cos(2 * math.pi * 5 * i / n[0]) * ones
    N = float(np.prod(n))
    dV = float(np.prod(h))
    sq = A[0] ** 2 / 2 + A[1] ** 2 / 2 + A[2] ** 2 + C[0] ** 2 / 2 + C[1] ** 2 / 2 + C[2] ** 2 / 2
    expect = 0.5 * sq * N * dV
    ek, ef, qt = O.energy(g, [])
    assert ek == 0.0 and qt == 0.0
    assert abs(ef - expect) < 1e-12 * expect


# ---------------------------------------------------- kinetic <-> field exchange
def test_langmuir_energy_exchange():
    """Cold plasma oscillation at omega_p: the kinetic energy and the field
    energy take turns, with equal maxima, and their sum stays constant to the
    percent level set by the half-step offset of the diagnostic."""
    nx, ny, h = 32, 2, 0.1
    dt = 0.95 * h / math.sqrt(2)
    g = O.Grid(2, (nx, ny), (h, h), dt, 1)
    ppx = 2
    xs = (np.arange(nx * ppx) + 0.5) * h / ppx
    ys = (np.arange(ny * ppx) + 0.5) * h / ppx
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    w = h * h / (ppx * ppx)
    k = 2 * math.pi / (nx * h)
    u = np.zeros((3, X.size))
    u[0] = 1e-3 * np.sin(k * X)
    sp = O.Species(-1.0, 1.0, np.stack([X, Y]), u, np.full(X.size, w))
    ek, ef = [], []
    for s in range(200):                          # ~2 plasma periods
        O.step(g, [sp], s * dt)
        e = O.energy(g, [sp])
        ek.append(e[0])
        ef.append(e[1])
    ek, ef = np.array(ek), np.array(ef)
    tot = ek + ef
    assert abs(ef.max() / ek.max() - 1.0) < 0.02
    assert (tot.max() - tot.min()) < 0.05 * ek.max()
    # both really exchange: each falls to a few percent of its maximum
    assert ek.min() < 0.05 * ek.max() and ef.min() < 0.05 * ef.max()


# ---------------------------------------------------------------- the laser
def _envelope(sig):
    """|analytic signal| of a real time series (FFT Hilbert transform)."""
    n = sig.size
    F = np.fft.fft(sig)
    hmul = np.zeros(n)
    hmul[0] = 1.0
    if n % 2 == 0:
        hmul[n // 2] = 1.0
        hmul[1:n // 2] = 2.0
    else:
        hmul[1:(n + 1) // 2] = 2.0
    return np.abs(np.fft.ifft(F * hmul))


def _record_laser(dim):
    lam = 2 * math.pi
    dx = lam / 16
    nx = 24
    ny = 128 if dim == 2 else 96
    nz = 96
    h = (dx, dx, dx)[:dim]
    n = (nx, ny, nz)[:dim]
    dt = 0.95 * dx / math.sqrt(dim)
    a0, w0 = 2.0, (2 * lam if dim == 2 else 1.5 * lam)
    tau = 4 * lam                                    # four cycles (omega = 1)
    yc = ny * dx / 2
    zc = nz * dx / 2 if dim == 3 else 0.0
    laser = O.Laser(a0=a0, w0=w0, tau=tau, omega=1.0, yc=yc, zc=zc)
    g = O.Grid(dim, n, h, dt, 1, absorb_x=True, laser=laser)
    probe = 6                                        # node column of E_y, x = 6 dx
    nst = int((tau + nx * dx) / dt) + 40
    rec = []
    for s in range(nst):
        O.step(g, [], s * dt)
        if dim == 2:
            rec.append(g.E[1][0, :, probe].copy())
        else:
            rec.append(g.E[1][nz // 2, :, probe].copy())
    t = (np.arange(nst) + 1) * dt                    # E after step s is at t_{s+1}
    return dict(rec=np.array(rec), t=t, x=probe * dx, dx=dx, dt=dt, a0=a0, w0=w0, tau=tau,
                yc=yc, ny=ny)


@pytest.mark.parametrize("dim", [2, 3])
def test_laser_on_the_grid(dim):
    r = _record_laser(dim)
    a0, w0, tau, dx = r["a0"], r["w0"], r["tau"], r["dx"]
    ys = (np.arange(r["ny"]) + 0.5) * dx              # E_y sits at y = (j + 1/2) dy
    jc = int(np.argmin(np.abs(ys - r["yc"])))
    s = r["t"] - r["x"]                               # retarded time at the probe
    axis = r["rec"][:, jc]
    env = _envelope(axis)
    inside = (s > 0.15 * tau) & (s < 0.85 * tau)
    # amplitude a0 at the centre of the envelope, a0 / 2 at a quarter (sin^2)
    i_mid = int(np.argmin(np.abs(s - tau / 2)))
    i_q1 = int(np.argmin(np.abs(s - tau / 4)))
    i_q3 = int(np.argmin(np.abs(s - 3 * tau / 4)))
    assert abs(env[i_mid] / a0 - 1.0) < 0.03
    assert abs(env[i_q1] / a0 - 0.5) < 0.03
    assert abs(env[i_q3] / a0 - 0.5) < 0.03
    # nothing before the pulse arrives or after it has passed (beyond the
    # grid's dispersive precursor and ringing)
    before = s < -2 * dx
    after = s > tau + 4 * dx
    assert np.max(np.abs(axis[before])) < 1e-3 * a0
    assert np.max(np.abs(axis[after])) < 0.03 * a0
    # carrier: zero crossings inside the pulse are pi / omega apart
    sig = axis[inside]
    z = np.nonzero(np.sign(sig[1:]) != np.sign(sig[:-1]))[0]
    tz = [s[inside][k] - sig[k] * (s[inside][k + 1] - s[inside][k]) / (sig[k + 1] - sig[k]) for k in z]
    period2 = np.mean(np.diff(tz))
    assert abs(period2 / math.pi - 1.0) < 0.01
    # transverse 1/e radius of the envelope at the centre of the pulse
    env_y = np.array([_envelope(r["rec"][:, j])[i_mid] for j in range(r["ny"])])
    prof = env_y / env_y.max()
    right = ys > r["yc"]
    yy, pp = ys[right], prof[right]
    k = int(np.nonzero(pp < math.exp(-1.0))[0][0])
    y_e = yy[k - 1] + (math.exp(-1.0) - pp[k - 1]) * (yy[k] - yy[k - 1]) / (pp[k] - pp[k - 1])
    assert abs((y_e - r["yc"]) / w0 - 1.0) < 0.03
